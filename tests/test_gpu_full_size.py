"""Parity at the stated sizes of the workload configurations (GPU).

Section 3 ("Input Instances") ranks random lists, lists with locality and
Euler tours of random trees; the configurations here take those shapes at
their full sizes:
  config 2  single lists, n = 2^24 .. 2^30, random / locality / identity
            order, unweighted (int32 ranks) and int32 weights in
            [-1000, 1000] (int64 ranks);
  config 3  a forest of 2^27 elements (16 lists of 2^22 plus lists of
            geometric length, mean 64, labels interleaved) and the Euler tour
            of a random recursive tree with 2^26 vertices (+-1 weights);
  config 4  1024 instances, sizes floor(2^U), U ~ U[8, 22], int64 weights in
            [0, 2^20), one CUDA graph, autotuned ruler fraction;
  config 5  served requests of 2^10 .. 2^26 elements (int64 weights).
(Config 1, a random list of 2^20, is compared element by element in
test_gpu_parity.py.)

Where the CPU oracle finishes in seconds (locality order, the forest, the
Euler tour, instances and requests up to 2^22) the GPU result is compared
with it element by element.  A random-order single list of 2^28 or 2^30 is
checked against its closed form instead: the element at list position k has
rank n-1-k, or the suffix sum of the weights from position k (the terminal's
weight excluded, Section 1.1), computed here with integer cumsum; that
determines every element.  Batches and requests too large for the oracle are
checked with the full recurrence rank[i] = rank[succ i] + w[i] and rank 0 at
every terminal, which for a valid input also determines the result, plus a
sample of whole instances against the oracle.
"""
import math

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_09318_gb300 as lr  # noqa: E402


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _device_random_order(n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randperm(n, device="cuda", generator=g, dtype=torch.int64)


def _succ_from_order(order):
    n = order.numel()
    s = torch.empty(n, dtype=torch.int64, device="cuda")
    s[order[:-1]] = order[1:]
    s[order[-1]] = order[-1]
    out = s.to(torch.int32)
    del s
    return out


def _check_recurrence(succ_global, weight, rank):
    """rank 0 at terminals, rank[i] = rank[succ i] + w(i) elsewhere (int64)."""
    n = succ_global.numel()
    idx = torch.arange(n, device="cuda", dtype=torch.int64)
    term = succ_global == idx
    r = rank.to(torch.int64)
    assert int(r[term].abs().sum()) == 0
    nt = ~term
    w = torch.ones(1, dtype=torch.int64, device="cuda") if weight is None else weight.to(torch.int64)[nt]
    assert bool((r[nt] == r[succ_global[nt]] + w).all())
    return int(term.sum())


@pytest.mark.parametrize("lg", [30, 29])
def test_config2_random_unweighted_full_size(lg):
    """Config 2 at 2^30 (the largest size) and 2^29 + 7 (ragged): every element
    against the closed form rank(order[k]) = n-1-k."""
    n = (1 << lg) + (7 if lg == 29 else 0)
    order = _device_random_order(n, 2000 + lg)
    succ = _succ_from_order(order)
    rank = lr.rank(succ)
    del succ
    got = rank[order]
    del rank
    want = torch.arange(n - 1, -1, -1, device="cuda", dtype=torch.int32)
    assert bool(torch.equal(got, want))


@pytest.mark.parametrize("n", [1 << 30, (1 << 30) + 1])
def test_log_form_size_limit(n):
    """The log form of level 0 takes lists up to 2^30 elements; one more
    element switches to the exchange form.  Both sides of that limit, every
    element against the closed form."""
    order = _device_random_order(n, 2300 + (n & 1))
    succ = _succ_from_order(order)
    rank = lr.rank(succ)
    del succ
    got = rank[order]
    del rank
    assert bool(torch.equal(got, torch.arange(n - 1, -1, -1, device="cuda", dtype=torch.int32)))


def test_ids_beyond_int32_int64_ranks():
    """A random list of 2^31 + 3 elements: successor ids above 2^31 (negative
    as int32 views of the uint32 array), int64 ranks (an int32 rank cannot
    hold n - 1), every element against the closed form."""
    n = (1 << 31) + 3
    # an affine permutation k -> (a k + b) mod n with gcd(a, n) = 1 (the
    # device's randperm sorts at most 2^31 - 1 keys); it scatters
    # consecutive list positions over the whole id range
    a, b = 2654435761, 12345
    assert math.gcd(a, n) == 1
    order = (torch.arange(n, device="cuda", dtype=torch.int64) * a + b) % n
    s = torch.empty(n, dtype=torch.int64, device="cuda")
    s[order[:-1]] = order[1:]
    s[order[-1]] = order[-1]
    succ = (s & 0xFFFFFFFF).to(torch.int32)      # the uint32 bit pattern
    del s
    rank = lr.rank(succ, rank_dtype=torch.int64)
    del succ
    got = rank[order]
    del rank
    assert bool(torch.equal(got, torch.arange(n - 1, -1, -1, device="cuda", dtype=torch.int64)))


def _weighted_closed_form(order, w):
    """Suffix sums of the link weights along the order, the terminal's weight
    excluded: rank(order[k]) = sum_{j=k}^{n-2} w[order[j]]."""
    wo = w[order].to(torch.int64)
    wo[-1] = 0
    return torch.flip(torch.cumsum(torch.flip(wo, [0]), 0), [0])


@pytest.mark.parametrize("wdt", [torch.int32, torch.int64])
def test_config2_random_weighted_2p28(wdt):
    """Config 2, weights uniform in [-1000, 1000] stored as int32 (and as
    int64), int64 ranks, random order at 2^28: every element against the
    suffix sums of the weights along the list (through the exchange form)."""
    n = 1 << 28
    order = _device_random_order(n, 2100)
    succ = _succ_from_order(order)
    g = torch.Generator(device="cuda")
    g.manual_seed(2101)
    w = torch.randint(-1000, 1001, (n,), device="cuda", generator=g, dtype=wdt)
    rank = lr.rank(succ, w)
    assert rank.dtype == torch.int64
    del succ
    want = _weighted_closed_form(order, w)
    assert bool(torch.equal(rank[order], want))


@pytest.mark.parametrize("kind", ["locality", "identity"])
def test_config2_ordered_weighted_2p28_against_oracle(kind):
    """Config 2, locality and identity orders at 2^28, unweighted and int32
    weighted: element by element against the oracle (tile-local contraction
    runs on these orders)."""
    n = 1 << 28
    succ = gen.list_of_order_kind(kind, n, 2200)
    d_succ = dev(succ)
    got = lr.rank(d_succ).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ))
    del got
    w = gen.weights_i32(n, 2201)
    got = lr.rank(d_succ, dev(w)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ, w, np.int64))


def test_config3_forest_2p27():
    """Config 3: 16 lists of 2^22 plus about a million lists of geometric
    length (mean 64), 2^27 elements, labels randomly interleaved; unweighted
    int32 ranks, element by element against the oracle."""
    succ, nlists = gen.forest(1 << 27, gen.config_seed(3), n_long=16, long_len=1 << 22, mean_short=64)
    assert nlists > 1_000_000
    got = lr.rank(dev(succ)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ))


def _depths(parent):
    """Depth of every vertex of a rooted tree (parent[0] = 0) by pointer
    doubling over the parent array: from the tree alone."""
    d = (np.arange(parent.shape[0]) > 0).astype(np.int64)
    a = parent.astype(np.int64).copy()
    while np.any(a != 0):
        d = d + d[a]
        a = a[a]
    return d


def test_config3_euler_tour_2p26():
    """Config 3: the Euler tour of a random recursive tree with 2^26 vertices
    (2^27 - 2 arcs, +1 down, -1 up, int32 ranks), element by element against
    the oracle, and the node depths read off the ranks against the depths
    computed from the tree: depth(v) = 2 - rank[down(v)],
    depth(parent v) = -rank[up(v)]."""
    V = 1 << 26
    parent = gen.random_recursive_tree(V, gen.config_seed(3, 1))
    succ, w = gen.euler_tour(parent)
    got = lr.rank(dev(succ), dev(w), rank_dtype=torch.int32).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.rank(succ, w, np.int32))
    depth = _depths(parent)
    v = np.arange(1, V)
    down, up = 2 * (v - 1), 2 * (v - 1) + 1
    np.testing.assert_array_equal(2 - got[down].astype(np.int64), depth[v])
    np.testing.assert_array_equal(-got[up].astype(np.int64), depth[parent[v]])


def test_config4_batch_1024_in_cuda_graph():
    """Config 4: 1024 random-order instances (about 4.3e8 elements), int64
    weights in [0, 2^20), autotuned, captured in a CUDA graph and replayed.
    Full recurrence over every instance on the device, and 24 whole instances
    (the largest among them) against the oracle."""
    k = 1024
    offsets, succ, w = gen.batch_instances(k, gen.config_seed(4), 8.0, 22.0)
    n = int(offsets[-1])
    assert n > 4.0e8
    d_off, d_succ, d_w = dev(offsets), dev(succ), dev(w)
    lr.autotune(succ=d_succ, weight=d_w, offsets=d_off, max_lists=k)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = torch.empty(lr.workspace_size(n, k, weighted=True, max_lists=k), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    kw = dict(out=out, max_lists=k, n_total=n, sync=False, stream=s, workspace=ws)
    with torch.cuda.stream(s):
        lr.rank_batch(d_off, d_succ, d_w, **kw)              # warm-up outside capture
    s.synchronize()
    assert lr.device_status(s) == 0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        lr.rank_batch(d_off, d_succ, d_w, **kw)
    out.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    assert lr.device_status(s) == 0
    del ws
    lens = torch.from_numpy(np.diff(offsets)).cuda()
    inst = torch.repeat_interleave(torch.arange(k, device="cuda"), lens)
    sg = d_off[inst] + (d_succ.to(torch.int64) & 0xFFFFFFFF)
    del inst
    assert _check_recurrence(sg, d_w, out) == k                # one terminal per instance
    del sg
    got = out.cpu().numpy()
    rng = np.random.default_rng(4001)
    pick = set(rng.choice(k, 23, replace=False).tolist()) | {int(np.argmax(np.diff(offsets)))}
    for j in sorted(pick):
        a, b = int(offsets[j]), int(offsets[j + 1])
        np.testing.assert_array_equal(got[a:b], oracle.rank(succ[a:b], w[a:b], np.int64))
    lr.autotune_clear()                                      # leave no tuned entry behind


@pytest.mark.parametrize("total", [(1 << 31) - 4, (1 << 31) + 4])
def test_batch_order_limit_2p31(total):
    """A batch of four unweighted instances of about 2^29 elements each, just
    below 2^31 elements in all (levels chased in element order, the largest
    size that takes it) and just above (per-CTA slices of ruler ids), int64
    ranks: every element against its instance's closed form.  Each instance
    is an affine order k -> (a k + b) mod m (gcd(a, m) = 1) of its local ids,
    so no permutation of 2^29 has to be drawn."""
    k = 4
    m = [total // k + (1 if j < total % k else 0) for j in range(k)]
    offsets = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(m, out=offsets[1:])
    a, b = 2654435761, 12345
    succ = torch.empty(total, dtype=torch.int32, device="cuda")
    for j in range(k):
        assert math.gcd(a, m[j]) == 1
        order = (torch.arange(m[j], device="cuda", dtype=torch.int64) * a + b) % m[j]
        loc = torch.empty(m[j], dtype=torch.int64, device="cuda")
        loc[order[:-1]] = order[1:]
        loc[order[-1]] = order[-1]
        succ[int(offsets[j]):int(offsets[j + 1])] = loc.to(torch.int32)
        del order, loc
    rank = lr.rank_batch(dev(offsets), succ, rank_dtype=torch.int64, max_lists=k)
    del succ
    for j in range(k):
        order = (torch.arange(m[j], device="cuda", dtype=torch.int64) * a + b) % m[j]
        got = rank[int(offsets[j]):int(offsets[j + 1])][order]
        assert bool(torch.equal(got, torch.arange(m[j] - 1, -1, -1, device="cuda", dtype=torch.int64))), j
        del order, got


def test_config5_served_requests_full_sizes():
    """Config 5: requests of 2^10 .. 2^26 elements, random or locality order,
    int64 weights, served by continuous batching under a 40 GB budget.  Each
    result equals the request ranked alone; requests up to 2^22 equal the
    oracle, larger ones satisfy the full recurrence."""
    _, sizes, kinds, seeds = gen.serving_trace(24, gen.config_seed(5), rate_per_s=1000.0)
    sizes[0] = 1 << 26                                       # the largest size is present
    reqs = []
    for m, kind, sd in zip(sizes, kinds, seeds):
        succ = gen.list_of_order_kind(kind, int(m), int(sd % (1 << 31)))
        reqs.append((succ, gen.weights_i64(int(m), int(sd % (1 << 31)) + 1)))
    srv = lr.Server(budget_bytes=40_000_000_000)
    tickets = [srv.submit(dev(s_), dev(w_)) for s_, w_ in reqs]
    for (succ, w), t in zip(reqs, tickets):
        out, _ = srv.wait(t)
        alone = lr.rank(dev(succ), dev(w))
        assert bool(torch.equal(out, alone))
        if succ.shape[0] <= (1 << 22):
            np.testing.assert_array_equal(out.cpu().numpy(), oracle.rank(succ, w, np.int64))
        else:
            assert _check_recurrence(dev(succ).to(torch.int64) & 0xFFFFFFFF, dev(w), out) == 1
    assert srv.stats()["completed"] == len(reqs)
    srv.close()
