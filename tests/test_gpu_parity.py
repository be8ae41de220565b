"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Hull index lists are compared element by element (bit-exact), and the
per-level partition counters are compared with the oracle's, which use the
same tie rule.  Sizes span several partition tiles, ragged tails and every
level kind (level 0, big-segment levels, the shared-memory finisher).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_09417_gb300 as v
    v.load()
    return v


@pytest.fixture(autouse=True)
def _default_config(vq):
    cfg = vq.vq_get_config()
    yield
    vq.vq_set_config(cfg)


def gpu_hull(vq, x, y):
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
    return vq.vq_hull2d(xd, yd).cpu().numpy()


def check(vq, x, y, stats=False):
    """The hull (with the configured pre-filter) equals the oracle's; with
    stats, the per-level counters of plain Alg. 1 (pre-filter off, restored
    afterwards) equal the oracle's too."""
    got = gpu_hull(vq, x, y)
    if stats:
        want, st = oracle.hull(x, y, stats=True)
    else:
        want = oracle.hull(x, y)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    if stats:
        pre = vq.vq_get_config().prefilter
        vq.vq_set_config(prefilter=0)
        try:
            assert np.array_equal(gpu_hull(vq, x, y), want)
            gs = vq.vq_last_stats()
        finally:
            vq.vq_set_config(prefilter=pre)
        L = st["levels"]
        assert gs["levels"] == L
        assert gs["read"] == st["read"]
        assert gs["written"] == st["written"]
        assert gs["segments"] == st["segments"]
    return got


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 5000, 70_001])
def test_distributions(vq, dist, n):
    x, y = synth.points(dist, n, 1000 + n)
    check(vq, x, y, stats=True)


@pytest.mark.parametrize("small_max", [2, 64, 1024])
@pytest.mark.parametrize("ppt", [4, 8, 16])
def test_tilings(vq, small_max, ppt):
    """Every tile size and small-segment threshold gives the same hull and
    the same per-level counts."""
    vq.vq_set_config(points_per_thread=ppt, small_max=small_max)
    for dist, n in (("disk", 300_000), ("circle", 50_000), ("square", 123_457)):
        x, y = synth.points(dist, n, 7)
        check(vq, x, y, stats=True)


def test_degenerate(vq):
    rng = np.random.default_rng(4)
    cases = []
    cases.append((np.array([]), np.array([])))
    cases.append((np.full(10_000, 3.0), np.full(10_000, -2.0)))       # coincident
    t = rng.permutation(50_000).astype(float)
    cases.append((t, 3 * t - 7))                                       # collinear
    cases.append((np.zeros(20_000), rng.random(20_000)))              # vertical line
    g = rng.integers(0, 50, (2, 200_000)).astype(float)
    cases.append((g[0], g[1]))                                         # grid with duplicates
    k = 6
    gx, gy = np.meshgrid(np.arange(k + 1.0), np.arange(k + 1.0))
    cases.append((np.tile(gx.ravel(), 500), np.tile(gy.ravel(), 500)))  # lattice, many copies
    par = rng.permutation(np.arange(-40_000, 40_000, dtype=float))
    cases.append((par, par * par))                                     # parabola: all vertices
    x, y = synth.points("disk", 100_000, 5)
    cases.append((np.concatenate([x, x]), np.concatenate([y, y])))     # every point twice
    cases.append((x * 2.0 ** 200, y * 2.0 ** -200))                    # outside the FP32 tier's range
    cases.append((x * 2.0 ** -300, y * 2.0 ** -300))                   # tiny magnitudes
    for x, y in cases:
        check(vq, x, y)


def test_config1_square_1e6(vq):
    x, y = synth.workload("square", 1_000_000)
    check(vq, x, y, stats=True)


@pytest.mark.parametrize("dist", ["square", "disk", "kuzmin", "circle"])
def test_full_size_1e8(vq, dist):
    """The 1e8-point workloads: complete verification of the hull (unique by
    its invariants) at full size, plus exact equality with the oracle where
    it finishes in seconds."""
    x, y = synth.workload(dist, 100_000_000)
    got = gpu_hull(vq, x, y)
    code, bad = oracle.verify(x, y, got)
    assert code == 0, (oracle.VERIFY_CODES.get(code), bad)
    if dist in ("square", "kuzmin", "disk"):
        assert np.array_equal(got, oracle.hull(x, y))


def test_nonfinite(vq):
    x, y = synth.points("disk", 10_000, 1)
    x[1234] = np.nan
    with pytest.raises(vq.VQError) as e:
        gpu_hull(vq, x, y)
    assert e.value.status == -2


def test_batched_matches_single(vq):
    x, y, offs, dists = synth.batched_sets(nsets=300, lo=1, hi=200_000, seed=9)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    od = torch.from_numpy(offs).cuda()
    hi, ho = vq.vq_hull2d_batched(xd, yd, od)
    hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
    for s in range(300):
        a, b = offs[s], offs[s + 1]
        want = oracle.hull(x[a:b], y[a:b])
        got = hi[ho[s]:ho[s + 1]]
        assert np.array_equal(got, want), s


def test_batched_empty_sets(vq):
    x, y = synth.points("square", 1000, 2)
    offs = np.array([0, 0, 10, 10, 1000, 1000], dtype=np.int64)
    hi, ho = vq.vq_hull2d_batched(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                                  torch.from_numpy(offs).cuda())
    hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
    for s in range(5):
        a, b = offs[s], offs[s + 1]
        assert np.array_equal(hi[ho[s]:ho[s + 1]], oracle.hull(x[a:b], y[a:b]))


def test_batched_mixed_tiers(vq):
    """Sets inside and outside the FP32 tier's range in one call: the
    partition kernel compiled with both tiers runs the pre-filter on the
    sets that have it and the FP64 tier on the others."""
    parts, dists = [], []
    for s, (dist, n, scale) in enumerate((("disk", 300_000, 1.0), ("square", 200_000, 2.0 ** 45),
                                           ("kuzmin", 250_000, 1.0), ("disk", 150_000, 2.0 ** 50),
                                           ("square", 400_000, 1.0))):
        x, y = synth.points(dist, n, 300 + s)
        parts.append((x * scale, y * scale))
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    np.cumsum([p[0].shape[0] for p in parts], out=offs[1:])
    x = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] for p in parts])
    hi, ho = vq.vq_hull2d_batched(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                                  torch.from_numpy(offs).cuda())
    hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
    for s in range(len(parts)):
        a, b = offs[s], offs[s + 1]
        assert np.array_equal(hi[ho[s]:ho[s + 1]], oracle.hull(x[a:b], y[a:b])), s


def test_host_entry_point(vq):
    x, y = synth.points("kuzmin", 200_000, 3)
    got = vq.vq_hull2d_host(x, y)
    assert np.array_equal(got, oracle.hull(x, y))


def test_lookback_timeout_is_reported(vq):
    """A tile that never publishes its look-back status makes its successors'
    bounded waits expire; the call reports VQ_ERR_TIMEOUT and the device
    stays usable."""
    x, y = synth.points("square", 400_000, 3)
    # prefilter off: level 0 then partitions all 400K points in ordered mode
    vq.vq_set_config(ordered=1, debug_drop_tile=2, timeout_ns=20_000_000, prefilter=0)
    with pytest.raises(vq.VQError) as e:
        gpu_hull(vq, x, y)
    assert e.value.status == -6
    vq.vq_set_config(debug_drop_tile=-1, timeout_ns=2_000_000_000)
    check(vq, x, y)


@pytest.mark.parametrize("ppt", [4, 8, 16])
def test_ordered_mode(vq, ppt):
    """Offsets by decoupled look-back (stable partition) give the same hull
    and per-level counts as the default atomic offsets."""
    vq.vq_set_config(ordered=1, points_per_thread=ppt)
    for dist, n in (("disk", 300_000), ("circle", 120_000), ("square", 1_000_000), ("kuzmin", 200_000)):
        x, y = synth.points(dist, n, 17)
        check(vq, x, y, stats=True)


@pytest.mark.parametrize("ppt", [4, 8, 16])
def test_all_points_on_hull(vq, ppt):
    """Point sets where every point is a hull vertex (circle samples of
    1e5-2e5 points): the exact tiers decide most classifications and
    farthest points at every level, in big segments of one to a few tiles."""
    vq.vq_set_config(points_per_thread=ppt)
    # set 150 of the 300-set batched case (seed 9): 185,768 circle points
    x, y = synth.points("circle", 185_768, (9 << 20) + 150)
    check(vq, x, y, stats=True)
    for n, seed in ((100_000, 1), (150_001, 2), (200_000, 3)):
        x, y = synth.points("circle", n, seed)
        check(vq, x, y, stats=True)


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()


@pytest.mark.parametrize("case", ["disk", "duplicates", "circle"])
def test_host_entry_pipelined(vq, case):
    """Pinned host inputs large enough for several chunks (here three) take
    the chunked path (copies overlapped with chunk hulls, then the hull of
    the chunk hulls): same answer as the oracle, including the lowest index
    among coincident points in different chunks and the fallback when chunk
    hulls are large."""
    n = (1 << 25) + 12345
    if case == "disk":
        x, y = synth.points("disk", n, 21)
    elif case == "duplicates":
        a, b = synth.points("square", n // 2 + 1, 22)
        x, y = np.concatenate([a, a])[:n], np.concatenate([b, b])[:n]
    else:
        x, y = synth.points("circle", n, 23)
    got = vq.vq_hull2d_host(_pinned(x), _pinned(y))
    if case == "circle":
        code, bad = oracle.verify(x, y, got)
        assert code == 0, (oracle.VERIFY_CODES.get(code), bad)
    else:
        assert np.array_equal(got, oracle.hull(x, y))


@pytest.mark.parametrize("shift", [0, 1])
def test_extreme_ties_within_pairs(vq, shift):
    """The lexicographic extremes repeated at both points of a 16-byte pair
    of the extreme pass (and at odd offsets): the lowest index represents
    them, at the start and at the turn of the hull."""
    rng = np.random.default_rng(31 + shift)
    n = 50_000
    x, y = rng.random(n) + 1.0, rng.random(n) + 1.0
    for base in (2 + shift, 1000 + shift, 4096 + shift):
        x[base:base + 2] = 0.5       # lex-min, twice in a row
        y[base:base + 2] = 1.5
    for base in (6 + shift, 2000 + shift, 8190 + shift):
        x[base:base + 2] = 2.5       # lex-max, twice in a row
        y[base:base + 2] = 1.25
    check(vq, x, y)
    # the same through a batched call whose sets start at odd offsets
    offs = np.array([0, 1, 333, n], dtype=np.int64)
    hi, ho = vq.vq_hull2d_batched(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(offs).cuda())
    hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
    for s in range(3):
        a, b = offs[s], offs[s + 1]
        assert np.array_equal(hi[ho[s]:ho[s + 1]], oracle.hull(x[a:b], y[a:b])), s


@pytest.mark.parametrize("dist,n", [("disk", 5_000_000), ("circle", 4_194_304), ("square", 6_000_001)])
def test_device_level_loop(vq, dist, n):
    """Levels >= 1 as one CUDA graph launch (a WHILE node repeating two
    levels on the device) give the same hull and per-level counts as the
    host-driven loop, and as the oracle; repeated calls reuse the graph."""
    x, y = synth.points(dist, n, 41)
    vq.vq_set_config(host_loop=1)
    check(vq, x, y, stats=dist != "circle")
    vq.vq_profile_read(reset=True)
    ref = gpu_hull(vq, x, y)
    ref_stats = vq.vq_last_stats()
    assert vq.vq_profile_read()["graph_launches"] == 0
    vq.vq_set_config(host_loop=0)
    for _ in range(2):
        vq.vq_profile_read(reset=True)
        got = gpu_hull(vq, x, y)
        p = vq.vq_profile_read()
        assert p["graph_launches"] == 1
        assert np.array_equal(got, ref)
        assert vq.vq_last_stats() == ref_stats
    if dist == "circle":
        code, bad = oracle.verify(x, y, got)
        assert code == 0, (oracle.VERIFY_CODES.get(code), bad)


def test_device_level_loop_batched(vq):
    """The batched path through the device-driven level loop: every set's
    hull equals the oracle's."""
    x, y, offs, dists = synth.batched_sets(nsets=64, lo=2000, hi=1_000_000, seed=43)
    assert offs[-1] >= 1 << 22
    vq.vq_profile_read(reset=True)
    hi, ho = vq.vq_hull2d_batched(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                                  torch.from_numpy(offs).cuda())
    assert vq.vq_profile_read()["graph_launches"] == 1
    hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
    for s in range(64):
        a, b = offs[s], offs[s + 1]
        assert np.array_equal(hi[ho[s]:ho[s + 1]], oracle.hull(x[a:b], y[a:b])), s


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_prefilter(vq, dist):
    """The level-0 pre-filter (the sieve drops the points certainly inside
    the chains of sampled extremes before level 0) leaves every hull
    unchanged and only removes points: level 0 reads no more points than
    plain Alg. 1, and far fewer on the square and the disk, where the chains
    cover most of the set.  The later levels see a subset of the plain
    run's points."""
    x, y = synth.points(dist, 2_000_000, 77)
    want = oracle.hull(x, y)
    vq.vq_set_config(prefilter=0)
    assert np.array_equal(gpu_hull(vq, x, y), want)
    plain = vq.vq_last_stats()
    vq.vq_set_config(prefilter=1)
    assert np.array_equal(gpu_hull(vq, x, y), want)
    filt = vq.vq_last_stats()
    assert plain["read"][0] == 2_000_000
    assert filt["read"][0] <= plain["read"][0]
    assert filt["written"][0] <= plain["written"][0]
    assert sum(filt["read"]) <= sum(plain["read"])
    if dist in ("square", "disk"):
        assert filt["read"][0] < 0.05 * plain["read"][0]


def test_prefilter_degenerate_candidates(vq):
    """Sets whose pre-filter candidates coincide, tie or fall on the base
    line: points on the hull's edges, a triangle with its interior, a
    diamond whose diagonal extremes are whole edges, duplicated corners."""
    rng = np.random.default_rng(12)
    cases = []
    t = rng.random(200_000)                       # triangle (0,0), (1,0), (0,1) and its interior
    u = rng.random(200_000)
    m = t + u < 1
    cases.append((np.concatenate([t[m], [0.0, 1.0, 0.0]]), np.concatenate([u[m], [0.0, 0.0, 1.0]])))
    s = rng.integers(-1000, 1001, 300_000).astype(float)   # diamond |x| + |y| <= 1000 on a lattice
    r = rng.integers(-1000, 1001, 300_000).astype(float)
    k = np.abs(s) + np.abs(r) <= 1000
    cases.append((s[k], r[k]))
    a, b = rng.random(150_000), rng.random(150_000)      # unit square, corners repeated
    cases.append((np.concatenate([a, [0, 0, 1, 1, 0, 1]]), np.concatenate([b, [0, 1, 0, 1, 0, 1]])))
    g = rng.integers(0, 3, (2, 100_000)).astype(float)   # 3x3 grid with heavy duplication
    cases.append((g[0], g[1]))
    for x, y in cases:
        check(vq, x, y)


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
def test_aos_entry_point(vq, dist):
    """Interleaved (x, y) pairs (PBBS's layout, Sec. 5.4): the same hull as
    the oracle's on the de-interleaved points, also from an odd starting
    offset (8-byte but not 16-byte aligned) and in a batch of sizes that
    leave ragged last tiles."""
    for n, seed in ((3, 1), (1000, 2), (70_001, 3), (1_000_003, 4)):
        x, y = synth.points(dist, n, 40 + seed)
        want = oracle.hull(x, y)
        xy = torch.from_numpy(np.stack([x, y], 1)).cuda()
        assert np.array_equal(vq.vq_hull2d_aos(xy).cpu().numpy(), want), (dist, n)
        # one value before the pairs: the array starts 8 bytes past a 16-byte boundary
        buf = torch.empty(2 * n + 1, dtype=torch.float64, device="cuda")
        buf[1:] = xy.reshape(-1)
        assert np.array_equal(vq.vq_hull2d_aos(buf[1:]).cpu().numpy(), want), (dist, n, "offset")
