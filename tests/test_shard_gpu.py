"""The multi-GPU exchange on the device, with one GPU: the library's int64
texel accumulator, viewed in place by torch (shard.device_view) and reduced
through NCCL (a one-rank group, so the all-reduce is the identity) plus the
sums of the other half of the photon budget, equals one pass over the whole
budget bit for bit; so do the objective and, added as integers, the exact
gradient sums of the two halves. This is the arithmetic of a two-rank
photon shard (shard.ShardedPass) run on one device."""
import socket

import numpy as np
import pytest

from paper_2310_02043_gb300 import _build, scenes, shard
from paper_2310_02043_gb300.lighttrace import Tracer, fixed_to_ints

pytestmark = pytest.mark.gpu

N, HITS, SEED = 1 << 20, 5, 31


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_photon_halves_add_up_through_the_accumulator_view():
    import torch
    import torch.distributed as dist
    _build.build()
    torch.cuda.set_device(0)
    tr = Tracer(0, torch.cuda.current_stream().cuda_stream)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
        T = tr.upload_scene(sc)
        tr.set_lights(L)
        target = scenes.random_weights(T, seed=3, scale=2.0).astype(np.float32) ** 2
        tr.set_target(target)
        # the whole budget in one pass
        tr.trace_forward(SEED, N, HITS)
        q_full = tr.texel_sums()
        O_full = tr.loss()
        g_full = tr.trace_adjoint(SEED + 1, N, HITS)
        f_full, G_full = tr.gradient_fixed()
        # the second half, as another rank would hold it
        tr.trace_forward(SEED, N, HITS, N // 2, N)
        q_b = torch.from_numpy(tr.texel_sums()).cuda()
        # the first half in the library's accumulator, then the exchange
        tr.trace_forward(SEED, N, HITS, 0, N // 2)
        ptr, _ = tr.texel_accumulator()
        view = shard.device_view(ptr, T)
        shard.allreduce_sum(view)            # NCCL over one rank: the identity, on the library's buffer
        view += q_b                          # what a second rank's all-reduce adds
        torch.cuda.synchronize()
        assert np.array_equal(tr.texel_sums(), q_full)
        assert tr.loss() == O_full           # same sums, same deterministic reduction
        # the adjoint over each half; the exact sums add up as integers
        tr.trace_adjoint(SEED + 1, N, HITS, 0, N // 2)
        f0, G0 = tr.gradient_fixed()
        tr.trace_adjoint(SEED + 1, N, HITS, N // 2, N)
        f1, G1 = tr.gradient_fixed()
        assert G0 == G1 == G_full            # G depends on the weights and lights only
        assert np.array_equal(fixed_to_ints(f0) + fixed_to_ints(f1), fixed_to_ints(f_full))
        assert np.all(np.abs(g_full) > 0)
    finally:
        dist.destroy_process_group()
        tr.close()
