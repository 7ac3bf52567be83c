"""Finite differences of the traced objective in the light's position over a
sweep of step sizes (the validation of the paper's Fig. 6): same seed for
every evaluation, Cornell box, point light, 3 hits. Small steps see the
discrete changes of paths (texel crossings, moving shadows) and large steps
the curvature; in between the adjoint gradient (Eq. 11, 14) must agree with
the finite difference. The sweep is printed for the record."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.lighttrace import Tracer

pytestmark = pytest.mark.gpu


def test_position_gradient_agrees_with_finite_differences_on_a_plateau():
    _build.build()
    sc = scenes.cornell_box(res=32)
    L = scenes.cornell_lights()
    target = oracle.forward(sc, scenes.perturb_lights(L, seed=1, pos_sigma=0.05), 101, 1 << 18, 3)["E"]
    tr = Tracer(0)
    tr.upload_scene(sc)
    tr.set_target(target.astype(np.float32))
    n, hits, seed = 1 << 22, 3, 7

    def O(lights):
        tr.set_lights(lights)
        tr.trace_forward(seed, n, hits)
        return tr.loss()

    O(L)
    g = tr.trace_adjoint(seed, n, hits)
    rows = []
    for axis in (0, 1, 2):
        for h in (1e-5, 1e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1):
            Lp, Lm = L.copy(), L.copy()
            Lp[0, 1 + axis] += h
            Lm[0, 1 + axis] -= h
            fd = (O(Lp) - O(Lm)) / (2 * h)
            rows.append((axis, h, fd, g[0, axis], abs(fd - g[0, axis]) / abs(g[0, axis])))
    tr.close()
    print("\naxis      h          FD        adjoint   rel diff")
    for r in rows:
        print(f"{'xyz'[r[0]]}   {r[1]:8.0e}  {r[2]:10.5g}  {r[3]:10.5g}  {r[4]:8.3g}")
    for axis in (0, 1, 2):
        best = min(r[4] for r in rows if r[0] == axis and 1e-3 <= r[1] <= 3e-2)
        assert best < 0.05, (axis, [r for r in rows if r[0] == axis])
