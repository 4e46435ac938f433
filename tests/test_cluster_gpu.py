"""GPU parity of the clustering stage (rvh_cluster: DBSCAN, rvh_gather)
against the FP64 oracle.  Every DBSCAN decision is an FP64 comparison made
in the same operation order on both sides, so labels, cluster counts, the
CSR permutation and offsets must be identical.  The full-size scene is
checked on sampled points by brute force (neighbour counts, border rule,
noise) and the whole pipeline -- clustering, gather, estimate -- against
the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2012_12618_gb300 import rvh, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    c = rvh.Context(0)
    yield c
    c.close()


def _cluster(torch, ctx, feats, eps, min_pts, max_clusters=None):
    f = np.ascontiguousarray(feats, dtype=np.float32)
    if f.ndim == 1:
        f = f[:, None]
    n, dim = f.shape
    dev = torch.device("cuda", 0)
    tf = torch.from_numpy(f.reshape(-1).copy()).to(dev)
    labels = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    mc = n if max_clusters is None else max_clusters
    offsets = torch.full((mc + 1,), -7, dtype=torch.int32, device=dev)
    nc = ctypes.c_int32(-1)
    rc = rvh.rvh_cluster(ctx.handle, tf, n, dim, eps, min_pts, labels, perm, offsets, mc, nc)
    torch.cuda.synchronize()
    return rc, int(nc.value), labels.cpu().numpy()[:n], perm.cpu().numpy()[:n], offsets.cpu().numpy()


def _csr(labels, n_clusters):
    keep = np.flatnonzero(labels >= 0)
    perm = keep[np.argsort(labels[keep], kind="stable")]
    offsets = np.zeros(n_clusters + 1, np.int64)
    np.cumsum(np.bincount(labels[keep], minlength=n_clusters), out=offsets[1:])
    return perm, offsets


def _check(torch, ctx, feats, eps, min_pts):
    rc, nc, lab, perm, off = _cluster(torch, ctx, feats, eps, min_pts)
    assert rc == rvh.RVH_OK, rvh.rvh_last_error(None)
    o = oracle.dbscan(np.asarray(feats, np.float32).astype(np.float64), eps, min_pts)
    assert nc == o["n_clusters"]
    assert np.array_equal(lab, o["labels"])
    p, offs = _csr(o["labels"], nc)
    assert np.array_equal(off[:nc + 1], offs)
    assert np.array_equal(perm[:offs[-1]], p)
    return lab


@pytest.mark.parametrize("dim,n,eps,min_pts", [(2, 3000, 0.35, 4), (3, 2500, 1.4, 5), (1, 2000, 0.004, 3),
                                               (4, 1500, 2.0, 6), (2, 1200, 0.25, 1)])
def test_random_sets(torch, ctx, dim, n, eps, min_pts):
    rng = np.random.default_rng(dim * 100 + n)
    f = rng.uniform(0, 10, (n, dim)) if dim != 3 else rng.normal(0, 4, (n, dim))
    _check(torch, ctx, f, eps, min_pts)


def test_scene_small(torch, ctx):
    s = synth.make_scene(synth.SCENES["scene_small"])
    lab = _check(torch, ctx, s.features(), 1.0, 4)
    assert lab.max() >= 40


def test_scene_medium(torch, ctx):
    s = synth.make_scene(synth.SCENES["scene"], n_objects=160, gen_seed=21)
    _check(torch, ctx, s.features(), 1.0, 4)


def test_edge_cases(torch, ctx):
    # empty, single point, all identical, eps = 0 with duplicates, NaN features, far-out values
    assert _cluster(torch, ctx, np.zeros((0, 2)), 1.0, 3)[:2] == (rvh.RVH_OK, 0)
    _check(torch, ctx, np.array([[1.0, 2.0]]), 0.5, 1)
    _check(torch, ctx, np.ones((50, 2)), 0.5, 4)
    g = np.repeat(np.arange(6.0)[:, None], 4, axis=0)
    _check(torch, ctx, np.concatenate([g, g], axis=1), 0.0, 3)
    f = np.random.default_rng(3).uniform(0, 5, (400, 2))
    f[7] = np.nan
    f[11, 0] = 3e38
    f[12] = [-3e38, 1e30]
    _check(torch, ctx, f, 0.4, 3)
    # too many clusters for the offsets given
    rc, nc, lab, _, off = _cluster(torch, ctx, np.arange(20.0)[:, None] * 10.0, 1.0, 1, max_clusters=5)
    assert rc == rvh.RVH_EINVAL and nc == 20 and np.array_equal(lab, np.arange(20))
    assert (off == -7).all()


@pytest.mark.parametrize("long_chain", [2048, 2049])
def test_csr_paths(torch, ctx, long_chain):
    # chains of points 1 apart (eps 1.0, min_pts 2), shuffled: the largest
    # cluster at and just past one block's sort capacity (2048 points)
    chains = [np.stack([np.arange(k, dtype=np.float64), np.full(k, 10.0 * c)], 1)
              for c, k in enumerate([long_chain, 700, 2047, 1])]
    f = np.concatenate(chains)
    f = f[np.random.default_rng(long_chain).permutation(f.shape[0])]
    lab = _check(torch, ctx, f, 1.0, 2)
    assert np.bincount(lab[lab >= 0]).max() == long_chain


def test_deterministic(torch, ctx):
    s = synth.make_scene(synth.SCENES["scene"], n_objects=256, gen_seed=22)
    a = _cluster(torch, ctx, s.features(), 1.0, 4)
    b = _cluster(torch, ctx, s.features(), 1.0, 4)
    for x, y in zip(a[2:], b[2:]):
        assert np.array_equal(x, y)


def test_full_scene_sampled(torch, ctx):
    s = synth.make_scene(synth.SCENES["scene"])
    f = s.features().astype(np.float64)
    rc, nc, lab, perm, off = _cluster(torch, ctx, s.features(), 1.0, 4)
    assert rc == rvh.RVH_OK
    assert off[0] == 0 and np.all(np.diff(off[:nc + 1]) > 0) and off[nc] == (lab >= 0).sum()
    assert np.array_equal(np.sort(perm[:off[nc]]), np.flatnonzero(lab >= 0))
    for c in range(0, nc, max(1, nc // 50)):
        members = perm[off[c]:off[c + 1]]
        assert (lab[members] == c).all() and np.all(np.diff(members) > 0)
    rng = np.random.default_rng(5)
    d2 = lambda p: ((f - f[p]) ** 2).sum(1)  # noqa: E731  (same sum order for 2 components)
    core_cache = {}

    def is_core(q):
        if q not in core_cache:
            core_cache[q] = int((d2(q) <= 1.0).sum()) >= 4
        return core_cache[q]

    for p in rng.choice(s.n_points, 150, replace=False):
        nb = np.flatnonzero(d2(p) <= 1.0)
        cores = [q for q in nb if is_core(q)]
        if len(nb) >= 4:      # core: every core neighbour in the same cluster
            assert all(lab[q] == lab[p] for q in cores) and lab[p] >= 0
        elif cores:           # border: the lowest-index core neighbour's cluster
            assert lab[p] == lab[min(cores)]
        else:
            assert lab[p] == -1


def test_pipeline_cluster_gather_estimate(torch, ctx):
    """Raw scene -> rvh_cluster -> rvh_gather -> rvh_estimate equals the
    oracle's DBSCAN followed by the oracle's estimate of the clusters."""
    s = synth.make_scene(synth.SCENES["scene_small"])
    dev = torch.device("cuda", 0)
    rc, nc, lab, perm, off = _cluster(torch, ctx, s.features(), 1.0, 4)
    assert rc == rvh.RVH_OK
    m = int(off[nc])
    tperm = torch.from_numpy(perm[:m].copy()).to(dev)
    taz, tdop = torch.from_numpy(s.azimuth).to(dev), torch.from_numpy(s.doppler).to(dev)
    gaz = torch.empty(m, dtype=torch.float32, device=dev)
    gdop = torch.empty(m, dtype=torch.float32, device=dev)
    assert rvh.rvh_gather(ctx.handle, tperm, m, taz, gaz, tdop, gdop) == rvh.RVH_OK
    g = G.run_rvh(ctx, gaz.cpu().numpy(), gdop.cpu().numpy(), off[:nc + 1], H=256, tau=0.1, seed=3)
    o_lab = oracle.dbscan(s.features().astype(np.float64), 1.0, 4)["labels"]
    p_o, off_o = _csr(o_lab, nc)
    o = G.run_oracle(s.azimuth[p_o], s.doppler[p_o], off_o.astype(np.int32), H=256, tau=0.1, seed=3)
    G.check_parity(G.compare(g, o, off_o), tau=0.1)
    # sanity against the scene's truth: the velocity along the line of sight
    # (a distant object spans a degree of azimuth, so its lateral component
    # is barely observable from one radar; its radial one is)
    err = []
    for c in range(nc):
        pts = p_o[off_o[c]:off_o[c + 1]]
        oid = np.bincount(s.object_id[pts] + 1).argmax() - 1
        if oid < 0:
            continue
        t = float(np.mean(s.azimuth[pts]))
        u = np.array([np.cos(t), np.sin(t)])
        err.append(abs(np.dot([g["vx"][c], g["vy"][c]], u) - np.dot(s.truth_v[oid], u)))
    assert np.median(err) < 0.05, np.median(err)


def test_nearest_neighbour_clustering_is_min_pts_one(torch, ctx):
    """Threshold nearest-neighbour clustering (single linkage cut at eps, one
    of the clustering choices Fig. 1 names) is DBSCAN with min_pts = 1: every
    point is a core point and the clusters are the connected components of
    the eps-graph.  rvh_cluster with min_pts = 1 equals scipy's connected
    components on a 16,895-point scene, cluster for cluster."""
    sparse = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    spatial = pytest.importorskip("scipy.spatial")
    s = synth.make_scene(synth.SCENES["scene"], n_objects=96, gen_seed=24)
    f = s.features()
    rc, nc, lab, perm, off = _cluster(torch, ctx, f, 0.8, 1)
    assert rc == rvh.RVH_OK and (lab >= 0).all()
    f64 = f.astype(np.float64)
    pairs = spatial.cKDTree(f64).query_pairs(0.8 + 1e-6, output_type="ndarray")
    d2 = ((f64[pairs[:, 0]] - f64[pairs[:, 1]]) ** 2).sum(1)
    pairs = pairs[d2 <= 0.8 * 0.8]  # the same test as the library: squared FP64 distance <= eps^2
    n = f.shape[0]
    g = sparse.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    ncc, cc = csgraph.connected_components(g, directed=False)
    assert nc == ncc
    # the same partition; clusters numbered by their smallest point index
    first = np.full(ncc, n)
    np.minimum.at(first, cc, np.arange(n))
    rank = np.empty(ncc, np.int64)
    rank[np.argsort(first)] = np.arange(ncc)
    assert np.array_equal(lab, rank[cc])

