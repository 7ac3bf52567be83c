"""Planted mistakes: each case copies the oracle, plants one plausible mistake
(a dropped term or factor, a wrong sign, a transposed operand or index, a
wrong constant), builds the copy on the CPU and checks that the pin meant to
catch that mistake fails on it. The oracle's own files are never changed:
the copy is compiled into a temporary directory and swapped in for the one
call."""
import contextlib
import ctypes
import os
import tempfile
import types

import pytest

import oracle
from oracle import surrogate as S
from tests import test_oracle_area as T_area
from tests import test_oracle_geometry as T_geo
from tests import test_oracle_gradient as T_grad
from tests import test_oracle_rng as T_rng
from tests import test_oracle_surrogate as T_sg
from tests import test_oracle_transport as T_tr


@contextlib.contextmanager
def planted_c(old, new):
    """The oracle's C library built from oracle.c with `old` replaced by `new`."""
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"the text to replace must occur once: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        c_path, so_path = os.path.join(d, "oracle_planted.c"), os.path.join(d, "liboracle_planted.so")
        with open(c_path, "w") as f:
            f.write(src.replace(old, new))
        oracle.compile_source(c_path, so_path)
        lib = ctypes.CDLL(so_path)
        oracle._declare(lib)
        oracle._load()                    # the real library first, so that it is what comes back
        saved = oracle._lib
        oracle._lib = lib
        try:
            yield
        finally:
            oracle._lib = saved


@contextlib.contextmanager
def planted_py(module, old, new):
    """Every name of `module` taken from a copy of its source with `old`
    replaced by `new`, so that whatever the pin calls runs the copy."""
    src = open(module.__file__).read()
    assert src.count(old) == 1, f"the text to replace must occur once: {old!r}"
    copy = types.ModuleType(module.__name__ + "_planted")
    copy.__file__ = module.__file__
    exec(compile(src.replace(old, new), module.__file__, "exec"), copy.__dict__)
    saved = {}
    for name, value in copy.__dict__.items():
        if not name.startswith("__") and hasattr(module, name):
            saved[name] = getattr(module, name)
            setattr(module, name, value)
    try:
        yield
    finally:
        for name, value in saved.items():
            setattr(module, name, value)


# (id, where: "c" for oracle.c or the Python module, text in the oracle,
#  planted text, the pin that must catch it)
CASES = [
    ("philox-multiplier", "c",
     "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
     "uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;",
     T_rng.test_philox_matches_triton_reference),
    ("spot-emission-cone", "c",
     "double c = 1.0 - u1 * (1.0 - L->co);",
     "double c = 1.0 - u1 * (1.0 - L->ci);",
     T_tr.test_spot_emission_is_uniform_in_the_outer_cone),
    ("spot-soft-edge-not-squared", "c",
     "    double s = (c - L->co) / (L->ci - L->co);\n    return s * s;",
     "    double s = (c - L->co) / (L->ci - L->co);\n    return s;",
     T_tr.test_spot_irradiance_on_plane_matches_quadrature),
    # (exchanging sqrt(u1) and sqrt(1 - u1) is no mistake: 1 - u1 is uniform
    # too, so the lobe is the same; the parity tests see that remapping)
    ("uniform-hemisphere-for-cosine-lobe", "c",
     "double r = sqrt(u1), phi = 2.0 * OR_PI * u2, z = sqrt(1.0 - u1);",
     "double r = sqrt(1.0 - u1 * u1), phi = 2.0 * OR_PI * u2, z = u1;",
     T_tr.test_cosine_directions_follow_the_cosine_lobe),
    ("albedo-dropped", "c",
     "phi *= rho;                                     /* Eq. 7",
     "phi *= 1.0;                                     /* Eq. 7",
     T_tr.test_bounce_flux_uses_the_albedo_of_the_surface_left),
    ("edge-function-transposed", "c",
     "float U = Cx * By - Cy * Bx;",
     "float U = Cx * Bx - Cy * By;",
     T_geo.test_closest_hit_matches_fp64_brute_force),
    ("chart-vertices-swapped", "c",
     "float u = h->b[0] * uv[0] + h->b[1] * uv[2] + h->b[2] * uv[4];",
     "float u = h->b[0] * uv[0] + h->b[1] * uv[4] + h->b[2] * uv[2];",
     T_geo.test_texels_of_direct_hits_match_analytic_plane_hits),
    ("inverse-square-gradient-sign", "c",
     "for (int k = 0; k < 3; ++k) out[k] = It * (n1[k] - 3.0 * c1 * u[k]) / (ell * ell * ell);",
     "for (int k = 0; k < 3; ++k) out[k] = It * (n1[k] + 3.0 * c1 * u[k]) / (ell * ell * ell);",
     T_grad.test_point_light_position_gradient_matches_closed_form),
    ("soft-edge-derivative-factor", "c",
     "double da_dc = 2.0 * (c - L->co) / (D * D);",
     "double da_dc = (c - L->co) / (D * D);",
     T_grad.test_spot_gradients_match_quadrature),
    ("area-cosine-derivative-sign", "c",
     "for (int i = 0; i < 3; ++i) g0[i] += k * (-(L->ns[i] + ct * u[i]) / ell);",
     "for (int i = 0; i < 3; ++i) g0[i] += k * ((L->ns[i] + ct * u[i]) / ell);",
     T_area.test_area_gradients_match_quadrature),
    ("intensity-derivative-factor", "c",
     "out[5] = L->p * L->omega * a_emit / (double)L->n_rays;",
     "out[5] = 2.0 * L->p * L->omega * a_emit / (double)L->n_rays;",
     T_grad.test_fd_exact_intensity_matches_adjoint_point_cornell),
    ("adjoint-throughput-dropped", "c",
     "g += io->w[t] * beta;",
     "g += io->w[t];",
     T_grad.test_fd_exact_intensity_matches_adjoint_point_cornell),
    ("point-emission-hemisphere", "c",
     "double c = 1.0 - 2.0 * u1;",
     "double c = 1.0 - u1;",
     T_tr.test_point_emission_is_uniform_on_the_sphere),
    ("area-emission-cosine-lobe", "c",
     "        double c = 1.0 - u1;\n",
     "        double c = sqrt(1.0 - u1);\n",
     T_area.test_emission_samples_the_rectangle_and_the_hemisphere),
    ("spot-solid-angle-of-the-inner-cone", "c",
     "o->omega = 2.0 * OR_PI * (1.0 - o->co);",
     "o->omega = 2.0 * OR_PI * (1.0 - o->ci);",
     T_tr.test_energy_closed_cube_spot_matches_cone_integral),
    ("intensity-not-halved", "c",
     "o->I = 0.5 * o->p * o->p;",
     "o->I = o->p * o->p;",
     T_tr.test_point_light_irradiance_on_plane_is_inverse_square),
    ("texel-area-of-one-axis", "c",
     "double a = tile_area[k] / ((double)res[2 * k] * (double)res[2 * k + 1]);",
     "double a = tile_area[k] / (double)res[2 * k];",
     T_tr.test_point_light_irradiance_on_plane_is_inverse_square),
    ("one-sided-triangles", "c",
     "if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;",
     "if (U < 0.0f || V < 0.0f || W < 0.0f) return 0;",
     T_geo.test_closest_hit_matches_fp64_brute_force),
    ("skip-tile-ignored", "c",
     "        if (s->tile[i] == skip_tile) continue;",
     "        if (0 && s->tile[i] == skip_tile) continue;",
     T_geo.test_skip_tile_excludes_the_tile_left),
    ("objective-area-weight-dropped", oracle,
     "O = 0.5 * float(np.sum(A * a * r * r))",
     "O = 0.5 * float(np.sum(a * r * r))",
     T_grad.test_loss_on_a_hand_computed_case),
    # the surrogate's oracle (oracle/surrogate.py)
    ("hash-prime", S,
     "PRIMES = (1, 2654435761, 805459861)",
     "PRIMES = (1, 2654435761, 805459863)",
     T_sg.test_hash_at_hand_computed_vertices),
    ("trilinear-weights-swapped", S,
     "w[..., c] *= f[..., a] if CORNERS[c, a] else 1.0 - f[..., a]",
     "w[..., c] *= 1.0 - f[..., a] if CORNERS[c, a] else f[..., a]",
     T_sg.test_encoding_reproduces_linear_fields_on_dense_levels),
    ("relu-dropped", S,
     "a.append(_round(np.maximum(z, 0.0), rounding))",
     "a.append(_round(z, rounding))",
     T_sg.test_network_matches_torch_autograd),
    ("relu-mask-dropped-in-backward", S,
     "dz = _round(da * (a[k] > 0.0), rounding)",
     "dz = _round(da, rounding)",
     T_sg.test_network_matches_torch_autograd),
    ("bf16-round-half-up", S,
     "b = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)",
     "b = (b + np.uint64(0x8000)) >> np.uint64(16) << np.uint64(16)",
     T_sg.test_bf16_matches_torch_and_ties_to_even),
    ("direct-term-inverse-cube-factor", S,
     "dD[:, 0:3] += (-2.0 * a * np.abs(cr) / r ** 3)[:, None] * u",
     "dD[:, 0:3] += (-3.0 * a * np.abs(cr) / r ** 3)[:, None] * u",
     T_sg.test_geometry_derivatives_against_central_differences),
    ("direction-derivative-sign", S,
     "P = (np.eye(3)[None] - u[:, :, None] * u[:, None, :]) / r[:, None, None]",
     "P = (np.eye(3)[None] + u[:, :, None] * u[:, None, :]) / r[:, None, None]",
     T_sg.test_geometry_derivatives_against_central_differences),
    ("surrogate-soft-edge-derivative-factor", S,
     "da_dcos = np.where(soft, 2.0 * s / (ci - co), 0.0)",
     "da_dcos = np.where(soft, s / (ci - co), 0.0)",
     T_sg.test_geometry_derivatives_against_central_differences),
    ("head-sigmoid-derivative", S,
     "return K, v * (1.0 - v) * D, R_SCALE * sigmoid(o[:, 1]), v",
     "return K, v * D, R_SCALE * sigmoid(o[:, 1]), v",
     T_sg.test_head_derivatives),
    ("adam-bias-correction-dropped", S,
     "vh = v / (1 - beta2 ** step)",
     "vh = v",
     T_sg.test_adam_matches_torch),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(case):
    _, where, old, new, pin = case
    ctx = planted_c(old, new) if where == "c" else planted_py(where, old, new)
    with ctx:
        with pytest.raises(AssertionError):
            pin()


def test_an_unmodified_copy_passes_every_pin():
    """The control: the same build and swap with nothing planted."""
    same = "float U = Cx * By - Cy * Bx;"
    pins = []
    for c in CASES:
        if c[1] == "c" and c[4] not in pins:
            pins.append(c[4])
    with planted_c(same, same):
        for pin in pins:
            pin()
    for module in (oracle, S):
        keep = "O = 0.5 * float(np.sum(A * a * r * r))" if module is oracle else "vh = v / (1 - beta2 ** step)"
        with planted_py(module, keep, keep):
            for c in CASES:
                if c[1] is module:
                    c[4]()
