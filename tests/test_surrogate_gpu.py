"""Irradiance surrogate on the GPU against its CPU oracle (oracle/surrogate.py),
through the C ABI of include/sg.h: hash encoding, the network's forward and
backward, training-batch gradients and the Adam step, the per-light response
and the design objective with its gradient.

Tolerances. The oracle applies the kernel's bf16 roundings at the same points
but accumulates in float64; the kernel accumulates in fp32 (at most 64 terms
per product, relative error ~1e-6). A bf16 rounding whose input lies within
that error of a rounding boundary can fall the other way (probability ~1e-3 per
value); one such flip moves a value by 2^-8 of itself and is damped by the
following layers. Hence: most elements agree to ~1e-5 of the array's scale,
and every element within 1-2 % of it."""
import numpy as np
import pytest

from oracle import surrogate as S
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.surrogate import Surrogate, split_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    _build.build()
    s = Surrogate(0)
    yield s
    s.close()


def _rng(seed):
    return np.random.default_rng(seed)


def _spot(rng, z=2.6):
    return np.array(scenes.spot_light((rng.uniform(1, 5), rng.uniform(0.5, 3.5), z), rng.uniform(0, 2 * np.pi),
                                      -np.pi / 2 + rng.uniform(-0.4, 0.4), 1.0, rng.uniform(0.3, 0.6), 1.0),
                    np.float64)


def _problem(seed, T, n_lights):
    rng = _rng(seed)
    x = np.column_stack([rng.uniform(0, 6, T), rng.uniform(0, 4, T), rng.uniform(0, 1.5, T)]).astype(np.float32)
    nt = rng.normal(size=(T, 3))
    nt = (nt / np.linalg.norm(nt, axis=1, keepdims=True)).astype(np.float32)
    area = (rng.uniform(0.5, 1.5, T) * 0.01).astype(np.float32)
    lo = np.array([-1.0, -1.0, -0.5], np.float32)
    ext = 8.0
    lights = np.array([_spot(rng) for _ in range(n_lights)])
    W = np.concatenate([S.bf16(rng.normal(size=s) * 0.25).ravel() for s in S.WEIGHT_SHAPES]).astype(np.float32)
    table = (rng.normal(size=(16, S.TABLE, 2)) * 0.5).astype(np.float32)
    return x, nt, area, lo, ext, np.float32(1.0 / ext), lights, W, table


def _close(got, ref, frac_exact, tol_all, name):
    scale = np.abs(ref).max()
    err = np.abs(np.asarray(got, np.float64) - ref)
    assert err.max() <= tol_all * scale, (name, err.max() / scale)
    assert np.mean(err <= 1e-4 * scale) >= frac_exact, (name, np.mean(err <= 1e-4 * scale))


def test_texel_centres_match_the_oracle():
    from paper_2310_02043_gb300.lighttrace import Tracer
    sc = scenes.office(seed=0, pitch=0.2)
    tr = Tracer(0)
    tr.upload_scene(sc)
    pos, nrm = tr.texel_centres()
    tr.close()
    p_or, n_or = S.texel_centres(sc)
    assert np.abs(pos - p_or).max() < 2e-5 * np.abs(p_or).max()
    assert np.abs(nrm - n_or).max() < 1e-6


def test_encoding(sg):
    x, nt, area, lo, ext, inv_ext, lights, W, table = _problem(1, 64, 1)
    sg.set_texels(x, nt, area, lo, ext)
    sg.set_params(W, table)
    rng = _rng(2)
    xn = rng.uniform(0, 1, size=(3000, 3)).astype(np.float32)
    xn[:8] = np.array([[0, 0, 0], [1, 1, 1], [np.float32(0.99999994)] * 3, [0.5, 0.25, 0.125], [1 / 16, 1 / 512, 0],
                       [0.3, 1.0, 0.0], [0.999, 0.001, 0.5], [1 / 3, 2 / 3, 0.2]], np.float32)
    got = sg.encode(xn)
    ref = S.encode(xn, table.astype(np.float64))
    assert np.abs(got - ref).max() < 1e-5 * np.abs(table).max() * 8


def test_network_forward_and_backward(sg):
    x, nt, area, lo, ext, inv_ext, lights, W, table = _problem(3, 64, 1)
    sg.set_texels(x, nt, area, lo, ext)
    sg.set_params(W, table)
    rng = _rng(4)
    B = 333                                     # ragged: not a multiple of 16
    X = rng.normal(size=(B, 64)).astype(np.float32)
    dO = rng.normal(size=(B, 16)).astype(np.float32)
    O, dX, dW = sg.network(X, dO)
    Wm = [w.astype(np.float64) for w in split_weights(W)]
    o_ref, cache = S.mlp_forward(X.astype(np.float64), Wm)
    dX_ref, dW_ref = S.mlp_backward(cache, Wm, dO.astype(np.float64))
    _close(O, o_ref, 0.97, 2e-2, "O")
    _close(dX, dX_ref, 0.97, 2e-2, "dX")
    for k, (a, b) in enumerate(zip(split_weights(dW), dW_ref)):
        _close(a, b, 0.9, 2e-2, f"dW{k}")
    assert np.array_equal(sg.network(X), O)      # forward alone gives the same rows


def _train_setup(sg, seed, T=500, S_=3, B=300):
    x, nt, area, lo, ext, inv_ext, lights, W, table = _problem(seed, T, S_)
    import torch
    rng = _rng(seed + 1)
    E_obs = rng.uniform(0, 0.3, size=(S_, T)).astype(np.float32)
    sg.set_texels(x, nt, area, lo, ext)
    sg.set_params(W, table)
    E_dev = torch.tensor(E_obs, device="cuda")
    sg.set_training_data(lights, E_dev)
    samples = np.column_stack([rng.integers(0, S_, B), rng.integers(0, T, B)]).astype(np.int32)
    return x, nt, area, lo, ext, inv_ext, lights, W, table, E_obs, E_dev, samples


def test_training_gradients(sg):
    x, nt, area, lo, ext, inv_ext, lights, W, table, E_obs, E_dev, samples = _train_setup(sg, 5)
    loss = sg.train_step(0, samples.shape[0], 0.0, samples)
    dW, dT = sg.gradients()
    Wm = [w.astype(np.float64) for w in split_weights(W)]
    loss_ref, dW_ref, dT_ref = S.train_gradients(table.astype(np.float64), Wm, samples, lights, E_obs, x,
                                                 nt.astype(np.float64), area, lo, ext, inv_ext)
    assert loss == pytest.approx(loss_ref, rel=2e-3)
    for k, (a, b) in enumerate(zip(split_weights(dW), dW_ref)):
        _close(a, b, 0.8, 3e-2, f"dW{k}")
    err = np.abs(dT - dT_ref)
    assert err.max() <= 3e-2 * np.abs(dT_ref).max()
    assert err.sum() <= 1e-2 * np.abs(dT_ref).sum()
    assert np.array_equal(dT != 0, dT_ref != 0) or np.mean((dT != 0) == (dT_ref != 0)) > 0.9999


@pytest.mark.parametrize("batch,drawn", [(300, False), (2000, True)])
def test_training_paths_agree(sg, batch, drawn):
    # tcgen05 (four 128-row tiles per CTA) and mma.sync (16 rows per warp) run
    # the same training step on the same samples, given or drawn on the
    # device from the seed and step: the loss and the gradients agree up to
    # the order of the fp32 sums and of the float atomics into the table.
    # 300 samples leave one warpgroup of the tcgen05 CTA without a tile.
    x, nt, area, lo, ext, inv_ext, lights, W, table, E_obs, E_dev, samples = _train_setup(sg, 21, B=batch)
    out = {}
    for tc in (True, False):
        sg.set_kernels(train_tcgen05=tc)
        sg.set_params(W, table)                  # restarts the step counter
        loss = sg.train_step(7, batch, 0.0, None if drawn else samples)
        out[tc] = (loss,) + sg.gradients()
    sg.set_kernels()
    (lt, dWt, dTt), (lm, dWm, dTm) = out[True], out[False]
    assert lt == pytest.approx(lm, rel=1e-4)
    assert np.abs(dWt - dWm).max() <= 1e-2 * np.abs(dWm).max()
    for k, (a, b) in enumerate(zip(split_weights(dWt), split_weights(dWm))):
        _close(a, b.astype(np.float64), 0.9, 1e-2, f"dW{k}")
    assert np.mean((dTt != 0) == (dTm != 0)) > 0.9999
    assert np.abs(dTt - dTm).max() <= 1e-2 * np.abs(dTm).max()
    assert np.abs(dTt - dTm).sum() <= 2e-3 * np.abs(dTm).sum()


def test_adam_step_moves_by_the_learning_rate(sg):
    x, nt, area, lo, ext, inv_ext, lights, W, table, E_obs, E_dev, samples = _train_setup(sg, 7)
    lr = 1e-3
    sg.train_step(0, samples.shape[0], lr, samples)
    W1, T1 = sg.params()
    Wm = [w.astype(np.float64) for w in split_weights(W)]
    _, dW_ref, _ = S.train_gradients(table.astype(np.float64), Wm, samples, lights, E_obs, x,
                                     nt.astype(np.float64), area, lo, ext, inv_ext)
    g = np.concatenate([d.ravel() for d in dW_ref])
    p_ref, _, _ = S.adam(W.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    big = np.abs(g) > 1e-2 * np.abs(g).max()
    assert big.sum() > 1000
    assert np.abs(W1[big] - p_ref[big]).max() < 1e-6 + 1e-6 * np.abs(W).max()
    # the next forward uses the updated weights
    X = _rng(8).normal(size=(32, 64)).astype(np.float32)
    o_new, _ = S.mlp_forward(X.astype(np.float64), [S.bf16(w) for w in split_weights(W1.astype(np.float64))])
    _close(sg.network(X), o_new, 0.95, 2e-2, "O after step")


def test_response_and_design(sg):
    import torch
    x, nt, area, lo, ext, inv_ext, lights, W, table = _problem(9, 2001, 3)
    lights = lights.copy()
    lights[:, 6] = [2.0, 1.2, 1.6]
    sg.set_texels(x, nt, area, lo, ext)
    sg.set_params(W, table)
    Wm = [w.astype(np.float64) for w in split_weights(W)]
    T64 = table.astype(np.float64)
    K = sg.response(lights[0])
    K_ref = S.response(T64, Wm, lights[0], x, nt.astype(np.float64), lo, ext, inv_ext)
    _close(K, K_ref, 0.97, 2e-2, "K")
    rng = _rng(10)
    target = rng.uniform(0, 0.5, x.shape[0]).astype(np.float32)
    alpha = rng.uniform(0.5, 1.0, x.shape[0]).astype(np.float32)
    E_out = torch.zeros(x.shape[0], device="cuda")
    O, g = sg.design(lights, torch.tensor(target, device="cuda"), torch.tensor(alpha, device="cuda"), E_out)
    O_ref, g_ref, E_ref = S.design_objective(T64, Wm, lights, x, nt.astype(np.float64), area.astype(np.float64),
                                             target.astype(np.float64), alpha.astype(np.float64), lo, ext, inv_ext)
    assert O == pytest.approx(O_ref, rel=5e-3)
    _close(E_out.cpu().numpy(), E_ref, 0.97, 2e-2, "E")
    assert np.all(g[:, 7] == 0)
    for k in range(7):
        col = g_ref[:, k]
        scale = np.maximum(np.abs(col), 0.05 * np.abs(col).max())
        assert np.all(np.abs(g[:, k] - col) <= 3e-2 * scale), (k, g[:, k], col)
    # alpha omitted means ones
    O1, _ = sg.design(lights, torch.tensor(target, device="cuda"))
    O1_ref = S.design_objective(T64, Wm, lights, x, nt.astype(np.float64), area.astype(np.float64),
                                target.astype(np.float64), np.ones(x.shape[0]), lo, ext, inv_ext)[0]
    assert O1 == pytest.approx(O1_ref, rel=5e-3)


def test_training_fits_a_smooth_response(sg):
    # E_obs = 0.7 D + 0.002: the model can represent it exactly (sigmoid(o0)
    # = 0.7, softplus(o1) = 0.2); a few hundred steps must cut the loss 10x
    import torch
    x, nt, area, lo, ext, inv_ext, lights, W0, table0 = _problem(11, 4000, 8)
    W, table = scenes.surrogate_init(0)
    E = np.stack([0.7 * S.geometry(L, x, nt, lo, ext)[2] + 0.002 for L in lights]).astype(np.float32)
    sg.set_texels(x, nt, area, lo, ext)
    sg.set_params(W, table)
    sg.set_training_data(lights, torch.tensor(E, device="cuda"))
    losses = [sg.train_step(1, 4096, 1e-2) for _ in range(300)]
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:5]), (losses[:5], losses[-5:])


@pytest.mark.parametrize("n_texels,powers", [(5003, [1.5, 1.0, 2.0, 0.7, 1.2]), (301, [1.3, 0.8]),
                                             (301, list(np.linspace(0.6, 1.8, 40)))])
def test_tensor_core_paths_agree(sg, n_texels, powers):
    # tcgen05 (TMEM accumulators, 128-row tiles, four per CTA) and mma.sync
    # (16 rows per warp) run the same network on the same bf16 inputs; only
    # the order of the fp32 sums differs. Up to 32 lights the tcgen05 design
    # runs as one fused kernel (2 lights: 64 texels per tile, 5 tiles, the
    # second CTA with three idle warpgroups); 40 lights take the four-kernel
    # tcgen05 path.
    import torch
    x, nt, area, lo, ext, inv_ext, lights, W, table = _problem(12, n_texels, len(powers))
    lights = lights.copy()
    lights[:, 6] = powers
    sg.set_texels(x, nt, area, lo, ext)
    sg.set_params(W, table)
    target = torch.tensor(np.random.default_rng(13).uniform(0, 0.5, x.shape[0]).astype(np.float32), device="cuda")
    out = {}
    for tc in (True, False):
        sg.set_kernels(tc)
        E = torch.zeros(x.shape[0], device="cuda")
        O, g = sg.design(lights, target, E_out=E)
        out[tc] = (sg.response(lights[1]), O, g, E.cpu().numpy())
    sg.set_kernels(True)
    Kt, Ot, gt, Et = out[True]
    Km, Om, gm, Em = out[False]
    _close(Kt, Km.astype(np.float64), 0.99, 1e-2, "K")
    _close(Et, Em.astype(np.float64), 0.99, 1e-2, "E")
    assert Ot == pytest.approx(Om, rel=1e-3)
    assert np.abs(gt - gm).max() <= 1e-2 * np.abs(gm).max()
    Wm = [w.astype(np.float64) for w in split_weights(W)]
    K_ref = S.response(table.astype(np.float64), Wm, lights[1], x, nt.astype(np.float64), lo, ext, inv_ext)
    _close(Kt, K_ref, 0.97, 2e-2, "K vs oracle")

