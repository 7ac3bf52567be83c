"""The wide BVH the library builds on the host (lt_build_bvh, the builder
lt_upload_scene runs), checked for the properties the traversal relies on,
without a GPU:

* the leaves partition the triangles, at most 3 to a leaf, and every
  triangle is reached from the root exactly once;
* a leaf slot's box is its triangles' bounds grown by the stated margin, an inner
  slot's box is bit for bit the union of its child node's slot boxes;
* empty slots are inverted boxes with the empty marker, inner_mask lists the
  inner slots, nodes are breadth-first and the depth is the number of levels;
* children sit in the slots that minimise the sum of
  -dot(child centre - node centre, slot direction), checked against the
  Hungarian assignment of scipy;
* a tree deeper than the traversal's 16 levels, an empty or a non-finite
  input is refused."""
import ctypes

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from paper_2310_02043_gb300 import _build, lighttrace, scenes

EMPTY = np.iinfo(np.int32).min
LEAF_MAX = 3
MAX_DEPTH = 16


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lighttrace.load_library()


def _boxes(nodes):
    lo = np.stack([nodes["lo_x"], nodes["lo_y"], nodes["lo_z"]], -1)     # [n, 8, 3]
    hi = np.stack([nodes["hi_x"], nodes["hi_y"], nodes["hi_z"]], -1)
    return lo, hi


def _check_tree(xyz, nodes, order, depth):
    xyz = np.asarray(xyz, np.float32).reshape(-1, 3, 3)
    n_tri, n_nodes = xyz.shape[0], nodes.shape[0]
    assert np.array_equal(np.sort(order), np.arange(n_tri))
    lo, hi = _boxes(nodes)
    child = nodes["child"]
    empty, inner = child == EMPTY, child >= 0
    leaf = ~empty & ~inner
    bits = ((nodes["inner_mask"][:, None] >> np.arange(8)) & 1).astype(bool)
    assert np.array_equal(bits, inner)
    assert np.all(lo[empty] > hi[empty]) and np.all(lo[~empty] <= hi[~empty])
    assert np.all((~empty).sum(1) >= 1)
    # breadth-first: node i's inner children take the next free indices
    kids = [np.sort(child[i][inner[i]]) for i in range(n_nodes)]
    assert np.array_equal(np.concatenate(kids + [np.zeros(0, np.int32)]), np.arange(1, n_nodes))
    level = np.zeros(n_nodes, np.int64)
    for i in range(n_nodes):
        level[child[i][inner[i]]] = level[i] + 1
    assert depth == level.max() + 1 <= MAX_DEPTH
    # leaves partition the leaf-ordered triangles
    code = -1 - child[leaf].astype(np.int64)
    first, count = code >> 2, (code & 3) + 1
    assert np.all(count <= LEAF_MAX)
    hits = np.zeros(n_tri, np.int64)
    for f, c in zip(first, count):
        hits[f:f + c] += 1
    assert np.all(hits == 1)
    # a leaf box is its triangles' bounds grown by pad = (max |coordinate| + 1)
    # 2^-19, in float (sums rounded to nearest, so the margin is pad within
    # half an ulp of the coordinate)
    pad = (np.abs(xyz).max() + np.float32(1.0)) * np.float32(2.0 ** -19)
    assert pad.dtype == np.float32
    for (i, k), f, c in zip(np.argwhere(leaf), first, count):
        v = xyz[order[f:f + c]].reshape(-1, 3)
        assert np.array_equal(lo[i, k], v.min(0) - pad) and np.array_equal(hi[i, k], v.max(0) + pad)
    # an inner slot's box is the union of its child's slot boxes, exactly
    for i, k in np.argwhere(inner):
        c = child[i, k]
        m = ~empty[c]
        assert np.array_equal(lo[i, k], lo[c][m].min(0)) and np.array_equal(hi[i, k], hi[c][m].max(0))
    # slot assignment: least sum of -dot(centre - node centre, direction)
    sign = np.array([[1.0 if (s >> a) & 1 else -1.0 for a in range(3)] for s in range(8)])
    extent = float(np.abs(xyz).max()) + 1.0
    for i in range(n_nodes):
        slots = np.flatnonzero(~empty[i])
        lo_i, hi_i = lo[i, slots].astype(np.float64), hi[i, slots].astype(np.float64)
        centre = 0.5 * (lo_i + hi_i)
        node_centre = 0.5 * (lo_i.min(0) + hi_i.max(0))
        cost = -(centre - node_centre) @ sign.T                               # [children, 8 slots]
        r, s = linear_sum_assignment(cost)
        assert cost[np.arange(len(slots)), slots].sum() <= cost[r, s].sum() + 1e-5 * extent


def _soup(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-2.0, 3.0, size=(n, 1, 3))
    return (c + rng.normal(0.0, 0.05, size=(n, 3, 3))).astype(np.float32)


@pytest.mark.parametrize("name", ["cornell", "office", "icosphere", "nested_shelf", "soup_1", "soup_5000"])
def test_tree_properties(lib, name):
    xyz = {"cornell": lambda: scenes.cornell_box(res=8).xyz,
           "office": lambda: scenes.office().xyz,
           "icosphere": lambda: scenes.icosphere(radius=1.0, subdiv=3, albedo=0.5).xyz,
           "nested_shelf": lambda: scenes.nested_shelf().xyz,
           "soup_1": lambda: _soup(1, 1),
           "soup_5000": lambda: _soup(5000, 2)}[name]()
    nodes, order, depth = lighttrace.build_bvh(xyz)
    _check_tree(xyz, nodes, order, depth)
    if name == "nested_shelf":
        assert 8 < depth <= MAX_DEPTH            # the kernels' two-word trail
    if name == "soup_1":
        assert nodes.shape[0] == 1 and depth == 1 and nodes["child"][0].tolist().count(EMPTY) == 7


def _shelf(n, ratio):
    """n strips in z = 0 whose widths shrink by `ratio` towards x = 0: the
    surface-area heuristic peels them off a few at a time, one level each."""
    tris = []
    for i in range(n):
        w0, w1 = ratio ** (i + 1), ratio ** i
        a, b, c, d = [w0, 0.2, 0], [w1, 0.2, 0], [w1, 0.8, 0], [w0, 0.8, 0]
        tris += [[a, b, c], [a, c, d]]
    return np.array(tris, np.float32)


def test_refusals(lib):
    nodes, order, depth = lighttrace.build_bvh(_shelf(135, 0.6))
    assert depth == MAX_DEPTH
    _check_tree(_shelf(135, 0.6), nodes, order, depth)
    with pytest.raises(lighttrace.LtError, match="LT_ERR_ARG"):
        lighttrace.build_bvh(_shelf(140, 0.6))                    # 17 levels
    bad = _soup(10, 3)
    bad[4, 1, 2] = np.nan
    with pytest.raises(lighttrace.LtError, match="LT_ERR_ARG"):
        lighttrace.build_bvh(bad)
    n_nodes, d = ctypes.c_int32(-1), ctypes.c_int32(-1)
    assert lib.lt_build_bvh(None, 0, None, 0, None, ctypes.byref(n_nodes), ctypes.byref(d)) == lighttrace.LT_ERR_ARG
    xyz = np.ascontiguousarray(scenes.office().xyz, np.float32)
    one = np.zeros(1, lighttrace.BVH_NODE_DTYPE)
    rc = lib.lt_build_bvh(xyz.ctypes.data_as(ctypes.c_void_p), xyz.shape[0], one.ctypes.data_as(ctypes.c_void_p), 1,
                          None, ctypes.byref(n_nodes), ctypes.byref(d))
    assert rc == lighttrace.LT_ERR_ARG and n_nodes.value > 1 and d.value >= 2     # counts still written
    assert lighttrace.BVH_NODE_DTYPE.itemsize == ctypes.sizeof(lighttrace.lt_bvh_node) == 240


def test_host_allocation_failure_is_a_status(lib, monkeypatch):
    """An exception inside the library (here an injected std::bad_alloc in
    the BVH build) comes back as LT_ERR_OOM, not as a crash, and the next
    call works."""
    xyz = np.ascontiguousarray(scenes.cornell_box(res=8).xyz, np.float32)
    n_nodes, d = ctypes.c_int32(-1), ctypes.c_int32(-1)
    monkeypatch.setenv("LT_FAULT_HOST_ALLOC", "1")
    rc = lib.lt_build_bvh(xyz.ctypes.data_as(ctypes.c_void_p), xyz.shape[0], None, 0, None, ctypes.byref(n_nodes),
                          ctypes.byref(d))
    assert rc == lighttrace.LT_ERR_OOM and n_nodes.value == -1
    monkeypatch.delenv("LT_FAULT_HOST_ALLOC")
    nodes, order, depth = lighttrace.build_bvh(xyz)
    _check_tree(xyz, nodes, order, depth)


# ---------------------------------------------------------------------------
# Compressed nodes (lt_compress_bvh): the form the kernels read when the BVH
# is not staged in shared memory.
# ---------------------------------------------------------------------------
FAR_SCALE = np.float32(1.0 + 2.0 * (3.0 * 2.0 ** -24) / (1.0 - 3.0 * 2.0 ** -24))


def _decode(cn):
    """Exact (float64) planes of compressed nodes: lo, hi [n, 8, 3]."""
    e = np.stack([(cn["meta"] >> (8 * a)) & 0xFF for a in range(3)], -1).astype(np.int64) - 142   # [n, 3]
    step = np.ldexp(1.0, e)[:, None, :]
    q = cn["q"].astype(np.float64)                                    # [n, 3, 16]
    origin = cn["origin"].astype(np.float64)[:, None, :]
    lo = origin + np.transpose(q[:, :, :8], (0, 2, 1)) * step
    hi = origin + np.transpose(q[:, :, 8:], (0, 2, 1)) * step
    return lo, hi, step[:, 0, :]


@pytest.mark.parametrize("name", ["cornell", "office", "nested_shelf", "soup_5000", "building_1"])
def test_compressed_nodes_contain_the_float_boxes(lib, name):
    xyz = {"cornell": lambda: scenes.cornell_box(res=8).xyz,
           "office": lambda: scenes.office().xyz,
           "nested_shelf": lambda: scenes.nested_shelf().xyz,
           "soup_5000": lambda: _soup(5000, 2),
           "building_1": lambda: scenes.building(floors=1).xyz}[name]()
    nodes, order, depth = lighttrace.build_bvh(xyz)
    cn = lighttrace.compress_bvh(nodes)
    assert np.array_equal(cn["child"], nodes["child"])
    assert np.array_equal(cn["meta"] >> 24, nodes["inner_mask"])
    flo, fhi = _boxes(nodes)
    lo, hi, step = _decode(cn)
    full = nodes["child"] != EMPTY
    f64lo, f64hi = flo.astype(np.float64), fhi.astype(np.float64)
    big = np.where(full[..., None], f64hi, -np.inf).max(1) - np.where(full[..., None], f64lo, np.inf).min(1)   # [n, 3]
    m = big * 2.0 ** -14
    # every box contains the float box widened by the margin, and is at most
    # one step wider on each side
    sel = full[..., None] & np.ones(3, bool)
    assert np.all((lo <= f64lo - m[:, None, :])[sel]) and np.all((hi >= f64hi + m[:, None, :])[sel])
    assert np.all((lo > f64lo - m[:, None, :] - step[:, None, :] - 1e-6 * (np.abs(f64lo) + 1))[sel])
    assert np.all((hi < f64hi + m[:, None, :] + step[:, None, :] + 1e-6 * (np.abs(f64hi) + 1))[sel])
    # the step is the smallest power of two whose 254 steps span the node
    origin = cn["origin"].astype(np.float64)
    span = np.where(full[..., None], f64hi, -np.inf).max(1) + m - origin
    assert np.all(254 * step >= span) and np.all((127 * step < span) | (step == 2.0 ** -126))
    # empty slots are inverted boxes
    q = cn["q"]
    for a in range(3):
        assert np.all(q[:, a, :8][~full] == 255) and np.all(q[:, a, 8:][~full] == 0)


def _fma32(a, b, c):
    """float32 fma emulated in float64 (the product of two float32 is exact in
    float64; the sum is rounded twice, within the tolerance used here)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_compressed_slab_test_is_conservative(lib):
    """The kernel's decode in float32 (planes as fma(1 + q 2^-15, E/d,
    (p - E - o)/d), the exit scaled by 1 + 2 gamma_3): for rays from points of
    the scene to points inside a child's triangle bounds, the child's box is
    entered no later and left no earlier than the point."""
    xyz = scenes.office().xyz
    nodes, order, depth = lighttrace.build_bvh(xyz)
    cn = lighttrace.compress_bvh(nodes)
    flo, fhi = _boxes(nodes)
    amax = float(np.abs(xyz).max())
    pad = (amax + 1.0) * 2.0 ** -19
    rng = np.random.default_rng(21)
    n_idx, k_idx = np.nonzero(nodes["child"] != EMPTY)
    pick = rng.integers(0, len(n_idx), 20000)
    n, k = n_idx[pick], k_idx[pick]
    # a point of the child's unpadded bounds, a ray origin anywhere in the room
    inner_lo, inner_hi = flo[n, k].astype(np.float64) + pad, fhi[n, k].astype(np.float64) - pad
    x = inner_lo + rng.uniform(0, 1, inner_lo.shape) * np.maximum(inner_hi - inner_lo, 0)
    lo_s, hi_s = xyz.reshape(-1, 3).min(0), xyz.reshape(-1, 3).max(0)
    o = rng.uniform(lo_s, hi_s, (len(n), 3)).astype(np.float32)
    d = x - o.astype(np.float64)
    dist = np.linalg.norm(d, axis=1)
    d = (d / dist[:, None]).astype(np.float32)
    d = np.where(np.abs(d) < 1e-30, np.copysign(np.float32(1e-30), d), d)
    inv = (np.float32(1.0) / d).astype(np.float32)
    meta, origin, q = cn["meta"][n], cn["origin"][n], cn["q"][n]
    tn = np.zeros(len(n), np.float32)
    tf = np.full(len(n), np.inf, np.float32)
    for a in range(3):
        E = np.ldexp(np.float32(1.0), ((meta >> (8 * a)) & 0xFF).astype(np.int64) - 127).astype(np.float32)
        S = (E * inv[:, a]).astype(np.float32)
        B = (((origin[:, a] - E).astype(np.float32) - o[:, a]).astype(np.float32) * inv[:, a]).astype(np.float32)
        qlo = (1.0 + q[np.arange(len(n)), a, k].astype(np.float64) * 2.0 ** -15).astype(np.float32)
        qhi = (1.0 + q[np.arange(len(n)), a, 8 + k].astype(np.float64) * 2.0 ** -15).astype(np.float32)
        t_lo, t_hi = _fma32(qlo, S, B), _fma32(qhi, S, B)
        near = np.where(d[:, a] < 0, t_hi, t_lo)
        far = np.where(d[:, a] < 0, t_lo, t_hi)
        tn = np.maximum(tn, near)
        tf = np.minimum(tf, far)
    tf = (tf * FAR_SCALE).astype(np.float32)
    ok = (tn.astype(np.float64) < dist * (1 - 2.0 ** -20)) & (tf.astype(np.float64) > dist * (1 + 2.0 ** -20))
    assert ok.all(), (np.count_nonzero(~ok), len(ok))


def test_compress_refusals(lib):
    nodes, order, depth = lighttrace.build_bvh(_soup(50, 4))
    bad = nodes.copy()
    k = int(np.nonzero(bad["child"][0] != EMPTY)[0][0])
    bad["lo_x"][0, k] = bad["hi_x"][0, k] + 1.0                 # an inverted box in a used slot
    with pytest.raises(lighttrace.LtError, match="LT_ERR_ARG"):
        lighttrace.compress_bvh(bad)
    bad = nodes.copy()
    bad["hi_y"][0, k] = np.nan
    with pytest.raises(lighttrace.LtError, match="LT_ERR_ARG"):
        lighttrace.compress_bvh(bad)
    out = np.zeros(1, lighttrace.CBVH_NODE_DTYPE)
    assert lib.lt_compress_bvh(None, 1, out.ctypes.data_as(ctypes.c_void_p)) == lighttrace.LT_ERR_ARG
    # nodes wider than the decode's range (about 2e6) are refused; 1e6 is fine
    for extent, ok in ((1.0e6, True), (4.0e6, False)):
        huge, _, _ = lighttrace.build_bvh(_soup(50, 4) * np.float32(extent / 5.0))
        if ok:
            lighttrace.compress_bvh(huge)
        else:
            with pytest.raises(lighttrace.LtError, match="LT_ERR_ARG"):
                lighttrace.compress_bvh(huge)
    assert lighttrace.CBVH_NODE_DTYPE.itemsize == ctypes.sizeof(lighttrace.lt_bvh_cnode) == 96
