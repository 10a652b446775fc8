"""Cases ranked by the debug build (run by test_gpu_debug_build.py in a
process of its own, with LR_DEBUG_LIB=1 so that the package loads
liblr_debug.so).  Every kernel path of the library runs once on a small
input; results must equal the oracle's and no index check may fail (a
failed check would come back as LR_ERR_INTERNAL)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402
import torch  # noqa: E402
import paper_2606_09318_gb300 as lr  # noqa: E402


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def check(name, got, want):
    np.testing.assert_array_equal(got, want, err_msg=name)
    print("ok", name, flush=True)


def main():
    assert lr.lib_path().endswith("liblr_debug.so"), lr.lib_path()
    n = (1 << 20) + 5
    succ = gen.random_list(n, 4900)
    w = gen.weights_i32(n, 4901)
    for tuning in ("", "log=1", "log=0", "spawn=1", "xchg=0", "algo=1"):
        os.environ["LR_TUNING"] = tuning
        check("unweighted " + tuning, lr.rank(dev(succ)).cpu().numpy(), oracle.rank(succ))
    for tuning in ("", "xchg=0", "spawn=1"):
        os.environ["LR_TUNING"] = tuning
        check("weighted " + tuning, lr.rank(dev(succ), dev(w)).cpu().numpy(), oracle.rank(succ, w, np.int64))
    os.environ["LR_TUNING"] = ""
    loc = gen.locality_list(n, 4902)
    check("contracted", lr.rank(dev(loc), dev(w)).cpu().numpy(), oracle.rank(loc, w, np.int64))
    r, t = lr.rank_outputs(dev(succ))[:2]
    check("outputs", r.cpu().numpy(), oracle.rank(succ))
    rng = np.random.default_rng(4903)
    lens = np.floor(2.0 ** rng.uniform(0, 15, size=200)).astype(np.int64)
    lens[rng.choice(200, size=20, replace=False)] = 0
    offsets = np.zeros(201, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    bs = np.concatenate([gen.random_list(int(m), 4904 + j).astype(np.uint32) if m else np.zeros(0, np.uint32)
                         for j, m in enumerate(lens)])
    bw = gen.weights_i64(int(offsets[-1]), 4905)
    want = oracle.rank_batch(offsets, bs, bw, np.int64)
    for tuning in ("ord=2,f0=8", "ord=1", "ord=0"):
        os.environ["LR_TUNING"] = tuning
        for ml in (0, 200):
            got = lr.rank_batch(dev(offsets), dev(bs), dev(bw), max_lists=ml).cpu().numpy()
            check("batch %s max_lists=%d" % (tuning, ml), got, want)
    os.environ["LR_TUNING"] = ""
    # invalid input keeps its own status: a list that skips its middle part,
    # which closes on itself (every in-degree at most one, one headless cycle)
    order = np.asarray(gen.random_order(n, 4906), dtype=np.int64)
    cyc = np.empty(n, dtype=np.int64)
    cyc[order[:-1]] = order[1:]
    cyc[order[-1]] = order[-1]
    cyc[order[n // 2 - 1]] = order[n - 1]
    cyc[order[n - 2]] = order[n // 2]
    assert oracle.STATUS_NAMES[oracle.rank_status(cyc.astype(np.uint32))[0]] == "CYCLE"
    for tuning in ("", "log=1"):
        os.environ["LR_TUNING"] = tuning
        try:
            lr.rank(dev(cyc.astype(np.uint32)))
            got = "LR_OK"
        except lr.LRError as e:
            got = e.name
        assert got == "LR_ERR_CYCLE", (tuning, got)
        print("ok cycle", tuning, flush=True)
    print("all ok", flush=True)


if __name__ == "__main__":
    main()
