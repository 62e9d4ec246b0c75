"""Property tests of the oracle (hypothesis, CPU): random grid shapes, NaN patterns, groups and
parameters, each checked against something fixed independently of the oracle's code --
brute-force components over the edges the vertex lists share, the zero motion of affine grids, the
fixed point of a constant normal field, numpy's first-maximum argmax, and the triangle count
over the quads' corners."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

import oracle  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None, derandomize=True)


def _vertex_lists(H, W):
    """Vertex indices of every GID: first = (p3, p2, p1), second = (p1, p4, p3) of quad (u, v)."""
    out = []
    for u in range(H - 1):
        for v in range(W - 1):
            p1, p2, p3, p4 = u * W + v, u * W + v + 1, (u + 1) * W + v + 1, (u + 1) * W + v
            out += [(p3, p2, p1), (p1, p4, p3)]
    return out


def _brute_components(H, W, G, tri_min):
    tris = _vertex_lists(H, W)
    n = len(tris)
    owner = {}
    for t, (a, b, c) in enumerate(tris):
        for e in ((a, b), (b, c), (c, a)):
            owner[e] = t
    lab = np.full(n, -1, np.int64)
    for s in range(n):                                    # BFS from the smallest unvisited GID
        if G[s] == 255 or lab[s] >= 0:
            continue
        lab[s] = s
        todo, members = [s], [s]
        while todo:
            t = todo.pop()
            a, b, c = tris[t]
            for x, y in ((a, b), (b, c), (c, a)):
                j = owner.get((y, x))
                if j is not None and lab[j] < 0 and G[j] == G[s]:
                    lab[j] = s
                    todo.append(j)
                    members.append(j)
        if tri_min > 0 and len(members) <= tri_min:
            lab[members] = -2                            # dropped, still visited
    lab[lab == -2] = -1
    return lab


@SETTINGS
@given(H=st.integers(2, 9), W=st.integers(2, 9), seed=st.integers(0, 2 ** 32 - 1), tri_min=st.integers(0, 5),
       n_groups=st.integers(1, 3))
def test_labels_are_the_brute_force_components(H, W, seed, tri_min, n_groups):
    rng = np.random.default_rng(seed)
    n = 2 * (H - 1) * (W - 1)
    G = rng.integers(0, n_groups, n).astype(np.uint8)
    G[rng.random(n) < 0.2] = 255
    np.testing.assert_array_equal(oracle.label(G, H, W, tri_min=tri_min), _brute_components(H, W, G, tri_min))


@SETTINGS
@given(H=st.integers(5, 10), W=st.integers(5, 10), seed=st.integers(0, 2 ** 32 - 1), kernel=st.sampled_from([3, 5]),
       lam=st.floats(0.0, 1.0), iters=st.integers(1, 3))
def test_affine_grids_do_not_move(H, W, seed, kernel, lam, iters):
    rng = np.random.default_rng(seed)
    o, A, B = rng.normal(0, 1, 3), rng.normal(0, 0.2, 3), rng.normal(0, 0.2, 3)
    u, v = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    P = o + u[..., None] * A + v[..., None] * B
    S = oracle.laplacian(P, kernel, lam, iters)
    scale = np.abs(P).max()
    assert np.abs(S - P).max() <= 1e-12 * max(scale, 1.0)


@SETTINGS
@given(H=st.integers(2, 8), W=st.integers(2, 8), seed=st.integers(0, 2 ** 32 - 1), kernel=st.sampled_from([3, 5]),
       sc=st.floats(0.01, 10.0), ss=st.floats(0.01, 10.0), iters=st.integers(1, 3))
def test_constant_normal_field_is_a_fixed_point(H, W, seed, kernel, sc, ss, iters):
    rng = np.random.default_rng(seed)
    n_tri = 2 * (H - 1) * (W - 1)
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    N = np.tile(nrm, (n_tri, 1))
    C = rng.normal(0, 1, (n_tri, 3))
    holes = rng.random(n_tri) < 0.2
    N[holes] = np.nan
    out = oracle.bilateral(C, N, H, W, kernel, sc, ss, iters)
    assert np.array_equal(np.isnan(out[:, 0]), holes)
    np.testing.assert_allclose(out[~holes], N[~holes], atol=1e-14)


@SETTINGS
@given(seed=st.integers(0, 2 ** 32 - 1), K=st.integers(1, 6), ang_min=st.floats(-1.0, 1.0))
def test_group_is_the_first_maximum_above_the_threshold(seed, K, ang_min):
    rng = np.random.default_rng(seed)
    n = 200
    N = rng.normal(size=(n, 3))
    N /= np.linalg.norm(N, axis=1)[:, None]
    nd = rng.normal(size=(K, 3))
    nd[rng.integers(0, K)] = nd[0]                        # a duplicated normal makes exact ties
    nd_unit = oracle.normalize_dominant(nd.astype(np.float32))
    m = (rng.random(n) < 0.9).astype(np.uint8)
    G, best, _ = oracle.classify(N, m, nd_unit, ang_min)
    dots = N @ nd_unit.T
    want = np.argmax(dots, axis=1)                        # numpy takes the first maximum
    want = np.where(dots.max(1) < ang_min, 255, want)
    want = np.where(m == 0, 255, want)
    np.testing.assert_array_equal(G, want.astype(np.uint8))


@SETTINGS
@given(H=st.integers(2, 12), W=st.integers(2, 12), seed=st.integers(0, 2 ** 32 - 1), frac=st.floats(0.0, 0.6))
def test_kept_triangles_are_those_with_three_valid_corners(H, W, seed, frac):
    rng = np.random.default_rng(seed)
    P = rng.normal(0, 1, (H, W, 3))
    bad = rng.random((H, W)) < frac
    P[bad] = np.nan
    m, _ = oracle.mask(P, P, 0.0)
    flat = bad.reshape(-1)
    want = [int(not (flat[a] or flat[b] or flat[c])) for a, b, c in _vertex_lists(H, W)]
    np.testing.assert_array_equal(m, want)
