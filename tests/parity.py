"""Parity helpers shared by the GPU tests: the CUDA path against the CPU
oracle on the same seeded inputs.

The two sides take the integer decisions of a segment (which triangle, which
texel) in float, but the CUDA path also computes the ray itself in float
while the oracle computes it in double and rounds it, so a small fraction of
photon paths part ways near triangle or texel edges. The helpers here find
those photons from the per-photon path records of both sides and account for
them exactly, so that everything else can be compared at the precision the
arithmetic allows:

  * ``check_every_texel``: every texel's irradiance, after removing the
    deposits of the photons whose paths parted (each side its own), agrees to
    ``rtol`` (1e-5) plus the rounding of the fixed-point quantum and of the
    float deposit values;
  * ``check_gradient``: the gradient as the CUDA path returns it, without any
    correction, agrees with the oracle's to ``raw_rtol`` of its largest
    component; then, with the parted photons' own terms exchanged, every
    component to ``rtol`` (against max(|g|, 1e-3 max |g|)). A parted photon's
    term differs wholesale, and a component that nearly cancels over the
    photons (a lateral position or an orientation slot) can be of the size
    of a few terms, so only the exchanged comparison is made per component.
"""
from __future__ import annotations

import numpy as np

import oracle


def light_sizes(n: int, n_lights: int) -> np.ndarray:
    """Photons per light: the budget split evenly, the first n mod L lights
    taking one extra (the contract of lt_trace_forward)."""
    return np.full(n_lights, n // n_lights, np.int64) + (np.arange(n_lights) < n % n_lights)


def light_of_photons(n: int, n_lights: int, begin: int, count: int) -> np.ndarray:
    ends = np.cumsum(light_sizes(n, n_lights))
    return np.searchsorted(ends, np.arange(begin, begin + count), side="right")


def emitted_flux(L, n: int, seed: int, photons, design: int = 0) -> np.ndarray:
    """Phi_r of the given photons (global indices of an n-photon budget),
    from the oracle's emission of each photon's own light."""
    sizes = light_sizes(n, L.shape[0])
    lights = np.searchsorted(np.cumsum(sizes), photons, side="right")
    return np.array([oracle.emit(L[l], int(sizes[l]), seed, int(p), design)[1] for p, l in zip(photons, lights)])


def check_every_texel(tr, sc, L, seed: int, n: int, hits: int, begin: int, end: int, q, scale: float,
                      design: int = 0, rtol: float = 1e-5, max_diverged: float = 1e-3) -> dict:
    """Every texel of the CUDA path's integer sums q (fixed-point scale
    `scale`) of photons [begin, end) against the oracle.

    `tr` must hold the same scene, lights and design word as the pass that
    produced q (its path record replays the pass). The photons whose
    (triangle, texel) sequence differs between the two path records are
    removed from each side with that side's own deposits: the oracle's from
    its record of the flux at every hit, the CUDA path's as Phi_r times the
    albedos of the surfaces its own path left (Eq. 7). What remains must
    agree texel by texel."""
    count = end - begin
    A = oracle.texel_areas(sc)
    ref = oracle.forward(sc, L, seed, n, hits, begin=begin, end=end, design=design, counts=True)
    tri_g, tex_g = tr.debug_paths(seed, n, hits, begin, count)
    tri_o, tex_o, phi_o = oracle.paths(sc, L, seed, n, hits, begin, count, design=design, flux=True)
    same = np.all(tri_g == tri_o, axis=1) & np.all(tex_g == tex_o, axis=1)
    div = np.nonzero(~same)[0]
    frac = len(div) / max(count, 1)
    assert frac <= max_diverged, f"{len(div)} of {count} photon paths parted"
    E_g = np.asarray(q, np.float64) / scale / A
    E_o = ref["E"].copy()
    removed = np.zeros(sc.n_texels, np.float64)       # deposits removed per texel, both sides
    if len(div):
        phi_r = emitted_flux(L, n, seed, begin + div, design)
        albedo = np.asarray(sc.albedo, np.float64)
        tg, xg = tri_g[div], tex_g[div]
        alive = tg >= 0
        rho = np.where(alive, albedo[np.maximum(tg, 0)], 1.0)
        beta = np.concatenate([np.ones((len(div), 1)), np.cumprod(rho, axis=1)[:, :-1]], axis=1)
        dep_g = phi_r[:, None] * beta
        E_g -= np.bincount(xg[alive], weights=dep_g[alive], minlength=sc.n_texels) / A
        xo, po = tex_o[div], phi_o[div]
        ok = xo >= 0
        E_o -= np.bincount(xo[ok], weights=po[ok], minlength=sc.n_texels) / A
        removed += np.bincount(xg[alive], minlength=sc.n_texels) + np.bincount(xo[ok], minlength=sc.n_texels)
    # Per deposit (kept, or removed with the other side's flux standing in
    # for the CUDA path's float one): the float flux differs from the double
    # one by a few ulps of Phi plus at most 1e-6 of the light's flux constant
    # (the spot's soft edge evaluated in float), and each deposit is rounded
    # to the fixed-point quantum 1 / scale.
    flux_max = float(np.max(np.abs(phi_o))) if phi_o.size else 0.0
    cnt = ref["count"].astype(np.float64) + removed
    tol = rtol * np.abs(E_o) + cnt * (2e-6 * flux_max + 1.0 / scale) / A
    err = np.abs(E_g - E_o)
    bad = np.nonzero(err > tol)[0]
    pos = E_o > 0
    rel = err[pos] / E_o[pos]
    info = dict(texels=int(sc.n_texels), lit=int(pos.sum()), diverged=int(len(div)), photons=int(count),
                max_rel=float(rel.max()) if rel.size else 0.0,
                max_err_over_tol=float((err / np.maximum(tol, 1e-300)).max()))
    assert len(bad) == 0, f"{len(bad)} of {sc.n_texels} texels beyond tolerance: {info}"
    info["touched"] = removed > 0        # texels that received a deposit of a parted photon (either side)
    info["count"] = ref["count"]
    return info


def check_gradient(tr, sc, L, seed: int, n: int, hits: int, w, g, g_ref, begin: int = 0, end: int | None = None,
                   design: int = 0, raw_rtol: float = 1e-3, rtol: float = 1e-3, max_diverged: float = 1e-3,
                   term_tol: float = 1e-2) -> dict:
    """The CUDA path's gradient g of photons [begin, end) against the oracle's
    g_ref from the same adjoint weights w.

    First the raw gate: g as returned within raw_rtol of max |g_ref| in every
    component (the componentwise error is reported). Then the per-photon terms
    from both path records: the photons whose paths parted must be rare, on
    agreeing paths the terms must agree (single terms within term_tol, 99.9 %
    within 1e-3; a first hit within rounding of a branch of dPhi/dp -- a
    spot's cone edges, cos_1 = 0 -- takes the branch in float on one side and
    in double on the other, so such terms may differ wholesale, but only
    rarely), the CUDA path's terms must sum to its aggregate, and with the
    parted and branch-edge photons' terms exchanged the aggregates must agree
    to rtol."""
    end = n if end is None else end
    count = end - begin
    g, g_ref = np.asarray(g, np.float64), np.asarray(g_ref, np.float64)
    den = np.maximum(np.abs(g_ref), 1e-3 * np.max(np.abs(g_ref)))
    raw = np.abs(g - g_ref) / den
    raw_norm = float(np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref)))
    info = dict(raw_norm_rel=raw_norm, raw_max_rel=float(raw.max()),
                raw_at=[int(i) for i in np.unravel_index(np.argmax(raw), raw.shape)])
    assert raw_norm <= raw_rtol, f"raw gradient beyond {raw_rtol} of its largest component: {info}"
    tri, tex, c = tr.debug_paths(seed, n, hits, begin, count, grads=True)
    tri_o, tex_o, c_o = oracle.paths(sc, L, seed, n, hits, begin, count, design=design, w=w)
    same = np.all(tri == tri_o, axis=1) & np.all(tex == tex_o, axis=1)
    info["diverged"] = int((~same).sum())
    assert 1.0 - same.mean() <= max_diverged, info
    col = np.maximum(np.abs(c_o).max(axis=0), 1e-300)
    diff = np.abs(c[same] - c_o[same]) / np.maximum(np.abs(c_o[same]), 1e-4 * col)
    off = diff.max(axis=1) > term_tol
    info["branch_edge"] = int(off.sum())
    assert off.mean() <= 1e-5 or off.sum() <= 1, f"{off.sum()} photon terms beyond {term_tol} (worst {diff.max():.3g})"
    assert np.quantile(diff.max(axis=1), 0.999) <= 1e-3
    lights = light_of_photons(n, L.shape[0], begin, count)
    g_sum = np.zeros_like(g)
    np.add.at(g_sum, lights, c)
    assert np.all(np.abs(g - g_sum) <= 1e-6 * np.maximum(np.abs(g_sum), np.abs(g_sum).max()))
    aside = ~same
    aside[np.nonzero(same)[0][off]] = True
    corr = np.zeros_like(g)
    np.add.at(corr, lights[aside], c[aside] - c_o[aside])
    rel = np.abs(g - corr - g_ref) / den
    info["corrected_max_rel"] = float(rel.max())
    assert np.all(rel <= rtol), f"corrected gradient beyond {rtol}: {info}"
    return info
