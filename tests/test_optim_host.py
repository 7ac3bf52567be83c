"""Host logic of the optimisation layer (autograd wiring, masks, recomputation,
checkpoint/resume, L-BFGS) with the CPU oracle standing in for the GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_02043_gb300 import optim, scenes
from tests.oracle_tracer import OracleTracer

N, HITS = 4096, 3


def _problem():
    sc = scenes.cornell_box(res=8)
    truth = scenes.make_lights([scenes.spot_light((0.45, 0.5, 0.9), 0.3, -1.3, 1.0, 0.4, 0.8)])
    target = oracle.forward(sc, truth, 99, 1 << 14, HITS)["E"]
    start = truth.copy()
    start[0, 1:4] += [0.06, -0.04, -0.05]
    start[0, 6] *= 1.1
    return sc, truth, target, start


def test_autograd_gradient_is_the_adjoint():
    sc, truth, target, start = _problem()
    tr = OracleTracer()
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=tr)
    rig = optim.LightRig(start)
    loss = prob.objective(rig, 5, 5)
    loss.backward()
    E = oracle.forward(sc, start, 5, N, HITS)["E"]
    O, w = oracle.loss(sc, E, target.astype(np.float32), np.ones(sc.n_texels))    # the target goes in as float
    g, _ = oracle.adjoint(sc, start, 5, N, HITS, w)
    assert float(loss.detach()) == pytest.approx(O, rel=1e-12)
    np.testing.assert_allclose(rig.params.grad.numpy(), g, rtol=1e-12, atol=1e-15)


def test_backward_recomputes_after_another_forward():
    sc, truth, target, start = _problem()
    tr = OracleTracer()
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=tr)
    rig_a, rig_b = optim.LightRig(start), optim.LightRig(truth)
    la = prob.objective(rig_a, 5, 6)
    prob.objective(rig_b, 7, 8)                     # overwrites the tracer's weights
    la.backward()
    # the adjoint ran on rig_a's lights after re-running rig_a's forward pass
    assert tr.calls[-2][0] == "forward" and tr.calls[-2][1] == 5 and np.allclose(tr.calls[-2][2], start)
    assert tr.calls[-1][0] == "adjoint" and tr.calls[-1][1] == 6 and np.allclose(tr.calls[-1][2], start)


def test_mask_keeps_unselected_parameters():
    sc, truth, target, start = _problem()
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=OracleTracer())
    rig = optim.LightRig(start, optimize=("x", "y", "z"))
    optim.adam(prob, rig, 3, lr=0.01)
    p = rig.params.detach().numpy()
    np.testing.assert_array_equal(p[:, 3:], start[:, 4:])
    assert np.any(p[:, :3] != start[:, 1:4])


def test_checkpoint_resume_repeats_the_uninterrupted_run(tmp_path):
    sc, truth, target, start = _problem()
    sched = optim.SeedSchedule(base=11)
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=OracleTracer())
    rig = optim.LightRig(start)
    losses, _ = optim.adam(prob, rig, 6, lr=0.02, schedule=sched)
    straight = rig.params.detach().clone()

    rig2 = optim.LightRig(start)
    l1, opt = optim.adam(prob, rig2, 3, lr=0.02, schedule=sched)
    path = str(tmp_path / "ckpt.pt")
    optim.save_checkpoint(path, rig2, opt, 3, sched)
    rig3 = optim.LightRig(start)
    opt3 = torch.optim.Adam([rig3.params], lr=0.02, betas=(0.9, 0.999))
    step, sched3 = optim.load_checkpoint(path, rig3, opt3)
    l2, _ = optim.adam(prob, rig3, 3, schedule=sched3, start_step=step, optimizer=opt3)
    assert torch.equal(rig3.params.detach(), straight)
    assert l1 + l2 == losses


def test_adam_recovers_a_perturbed_light():
    sc, truth, target, start = _problem()
    prob = optim.LightingProblem(sc, target, photons=1 << 14, hits=HITS, tracer=OracleTracer())
    # position and intensity were both perturbed, so both are optimised
    rig = optim.LightRig(start, optimize=("x", "y", "z", "p_int"))
    err0 = np.linalg.norm(start[0, 1:4] - truth[0, 1:4])
    perr0 = abs(start[0, 6] - truth[0, 6])
    losses, _ = optim.adam(prob, rig, 40, lr=0.005, schedule=optim.SeedSchedule(base=3))
    p = rig.params.detach().numpy()[0]
    assert np.linalg.norm(p[:3] - truth[0, 1:4]) < 0.6 * err0
    assert abs(p[5] - truth[0, 6]) < 0.5 * perr0
    assert np.mean(losses[-5:]) < 0.2 * losses[0]


def test_lbfgs_decreases_a_fixed_seed_objective():
    sc, truth, target, start = _problem()
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=OracleTracer())
    rig = optim.LightRig(start, optimize=("p_int", "theta_in"))
    trace = optim.lbfgs(prob, rig, max_iter=6, seed=4)
    assert trace[-1] < 0.5 * trace[0]


def test_seed_schedule():
    assert optim.SeedSchedule(base=5, correlated=True).seeds(2) == (5 + 2 * 7919,) * 2
    assert optim.SeedSchedule(base=5).seeds(0) == (5, 6)
    assert optim.SeedSchedule(base=5, fixed=True).seeds(9) == (5, 6)


def test_metrics_log_writes_one_line_per_step(tmp_path):
    import json
    sc, truth, target, start = _problem()
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=OracleTracer())
    rig = optim.LightRig(start, optimize=("x", "y", "z", "p_int"))
    schedule = optim.SeedSchedule(base=3)
    path = str(tmp_path / "run.jsonl")
    log = optim.MetricsLog(path, schedule)
    losses, _ = optim.adam(prob, rig, 3, lr=0.01, schedule=schedule, callback=log)
    log.close()
    rows = [json.loads(l) for l in open(path)]
    assert [r["step"] for r in rows] == [0, 1, 2]
    assert [r["loss"] for r in rows] == losses
    assert [tuple(r["seeds"]) for r in rows] == [schedule.seeds(k) for k in range(3)]
    assert set(rows[0]["grad_norm"]) == {"x", "y", "z", "p_int"} and rows[0]["grad_norm"]["x"] > 0
    assert rows[0]["t_s"] <= rows[1]["t_s"] <= rows[2]["t_s"]


def test_scaled_units():
    # params hold p / scale: the objective sees the physical parameters, the
    # gradient with respect to params is dO/dp x scale, and one Adam step
    # moves each column by about lr x its scale
    sc, truth, target, start = _problem()
    scale = [0.3, 0.3, 0.3, 0.1, 0.1, 0.2, 0.05, 1.0]
    prob = optim.LightingProblem(sc, target, photons=N, hits=HITS, tracer=OracleTracer())
    rig = optim.LightRig(start, scale=scale)
    np.testing.assert_allclose(rig.lights(), start, rtol=1e-15)
    loss = prob.objective(rig, 5, 5)
    loss.backward()
    plain = optim.LightRig(start)
    prob.objective(plain, 5, 5).backward()
    np.testing.assert_allclose(rig.params.grad.numpy(), plain.params.grad.numpy() * np.array(scale), rtol=1e-12)
    before = rig.lights()[0, 1:9].copy()
    optim.adam(prob, rig, 1, lr=0.01, schedule=optim.SeedSchedule(base=5, fixed=True))
    moved = np.abs(rig.lights()[0, 1:9] - before)
    for j in (0, 1, 2, 5, 6):        # optimised columns with a gradient: Adam's first step is lr x scale
        assert moved[j] == pytest.approx(0.01 * scale[j], rel=1e-6), j
    assert moved[7] == 0.0
    with pytest.raises(ValueError):
        optim.LightRig(start, scale=[1.0] * 7)
