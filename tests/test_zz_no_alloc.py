"""lt_loss_static: the objective for callers that cannot allocate device memory.

Code that runs inside another framework's memory pool, or on a device at its
memory budget, cannot call cudaMalloc; it gets the objective and the adjoint
weights from buffers it owns through lt_loss_static, whose only scratch is a
fixed array inside the library. This
file checks two calls in a row against lt_loss (the entry point that
allocates), on different targets, so a stale scratch array would show, and
that a call leaves the device's free memory unchanged."""
import numpy as np
import pytest

from paper_2310_02043_gb300 import _build, lighttrace, scenes
from paper_2310_02043_gb300.lighttrace import LtError, Tracer

pytestmark = pytest.mark.gpu

N, HITS = 1 << 18, 5


def test_static_loss_matches_lt_loss_on_two_calls():
    import torch
    _build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    tr = Tracer(0, stream)
    try:
        T = tr.upload_scene(sc)
        tr.set_lights(L)
        tr.trace_forward(3, N, HITS)
        q_ptr, scale = tr.texel_accumulator()
        area = torch.empty(T, dtype=torch.float32, device="cuda")
        tr.texel_areas(out=area)
        E_ref = torch.empty(T, dtype=torch.float32, device="cuda")
        tr.irradiance(out=E_ref)
        rng = np.random.default_rng(0)
        for call in range(2):
            factor = rng.uniform(0.5, 1.5, T).astype(np.float32)
            target = torch.from_numpy(E_ref.cpu().numpy() * factor).cuda()
            alpha = torch.from_numpy(rng.uniform(0.5, 1.5, T).astype(np.float32)).cuda()
            # the entry point that allocates
            tr.set_target(target, alpha)
            O_ref = tr.loss()
            g_ref = tr.trace_adjoint(4, N, HITS)
            # the one that does not
            w = torch.full((T,), float("nan"), dtype=torch.float32, device="cuda")
            E = torch.full((T,), float("nan"), dtype=torch.float32, device="cuda")
            O = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            lighttrace.loss_static(0, stream, q_ptr, scale, area, target, w, O, alpha=alpha, E_out=E)
            torch.cuda.synchronize()
            # the two sums differ only in the order of their double additions
            assert abs(O.item() - O_ref) <= 1e-12 * abs(O_ref), (call, O.item(), O_ref)
            assert torch.equal(E, E_ref)
            # identical weights give the identical (deterministic) adjoint
            tr.set_adjoint_weights(w)
            assert np.array_equal(tr.trace_adjoint(4, N, HITS), g_ref)
        # with its kernels loaded and its scratch array found by the calls
        # above, a call allocates no device memory: the device's free memory
        # and torch's allocation count are the same before and after it
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info(0)[0], torch.cuda.memory_allocated(0)
        lighttrace.loss_static(0, stream, q_ptr, scale, area, target, w, O, alpha=alpha, E_out=E)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(0)[0] == free0
        assert torch.cuda.memory_allocated(0) == alloc0
        # a shorter prefix after a full-length call: every block partial it
        # reads must be its own, not one left by the longer call; checked
        # against a float64 sum on the host over the same prefix
        n = T - 4096 - 7
        q = tr.texel_sums()
        lighttrace.loss_static(0, stream, q_ptr, scale, area[:n], target[:n], w[:n], O, alpha=alpha[:n])
        torch.cuda.synchronize()
        A = area[:n].cpu().numpy().astype(np.float64)
        r = q[:n].astype(np.float64) * (1.0 / scale) / A - target[:n].cpu().numpy().astype(np.float64)
        a = alpha[:n].cpu().numpy().astype(np.float64)
        O_host = 0.5 * float(np.sum(A * a * r * r))
        assert abs(O.item() - O_host) <= 1e-12 * O_host, (O.item(), O_host)
        # inputs beyond the fixed scratch array are refused before any launch
        big = torch.zeros(lighttrace.LOSS_STATIC_MAX_TEXELS + 1, dtype=torch.float32, device="cuda")
        with pytest.raises(LtError):
            lighttrace.loss_static(0, stream, q_ptr, scale, big, big, big, O)
    finally:
        tr.close()
