"""The stress workload with one packet per flow, as an overload case: the
g=1024, r=4, k=18 sketch (2 x 128 MiB of DHLA) fed 2^30 pairs of Zipf(1.0)
sources over 2^28 hosts and destinations over 2^30, half of them planted.
Each estimator then holds about 2^11 distinct peers of the natural traffic
alone, every one of them is hot (z_0 well below g e^(-theta/g)), and K
covers almost the whole key space, far above cand_cap.  Both sides must
flag the overload the same way: the same DHLA bits, row statistics, hot
counts and psi, and |K| reported as cand_cap + 1.

The window is drawn as 32 parts of 2^25 pairs from consecutive seeds (each
part a window of the same recipe), in parallel processes, which also run
the oracle's Algorithm 1 on their part; the parts' DHLAs are ORed (the
DHLA of the whole stream) before the oracle's close."""
import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu

SEED = 0x5EED5005
PARTS = 32
PART_PAIRS = 1 << 25


def _part(i):
    """Worker: draw part i and run the oracle's Algorithm 1 on it; returns
    (i, its pairs, its DHLA)."""
    import oracle as O
    from paper_1803_11449_gb300 import traffic as T
    w = T.WORKLOADS["stress"].with_(pkts_per_flow=1)
    win = T.make_window(w, T.window_seed(5) + 0x100000 * (i + 1), n=PART_PAIRS)
    op = O.params_from(w.sketch(), seed=SEED)
    grid = O.new_grid(op)
    O.update(op, grid, win.pairs)
    return i, win.pairs, grid


def test_stress_sketch_one_packet_per_flow_overloads_identically(O):
    import multiprocessing as mp
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd

    w = T.WORKLOADS["stress"].with_(pkts_per_flow=1)
    n = PARTS * PART_PAIRS
    dev = torch.empty(2 * n, dtype=torch.int32, device="cuda")
    og = None
    with mp.get_context("spawn").Pool(min(PARTS, mp.cpu_count() or 1)) as pool:
        for i, pairs, g in pool.imap_unordered(_part, range(PARTS)):
            dev[2 * i * PART_PAIRS:2 * (i + 1) * PART_PAIRS] = torch.from_numpy(pairs.reshape(-1).view(np.int32)).cuda()
            if og is None:
                og = g
            else:
                og |= g
    p = sd.params_for(w, SEED, cuda_stream=torch.cuda.current_stream().cuda_stream)
    h = sd.sd_create(p)
    try:
        sd.sd_update(h, dev)
        del dev
        grid = np.concatenate([sd.sd_get_grid(h, d) for d in range(p.dirs)])
        rep = sd.sd_close_window(h)
    finally:
        sd.sd_destroy(h)
    assert np.array_equal(grid, og), "DHLA bits differ"
    op = O.params_from(w.sketch(), seed=SEED)
    ref = O.close_window(op, og)
    cap = 1 << 20
    assert ref["flags"] == [O.FLAG_OVERLOAD_CANDS] * 2
    assert [rep.dir_flags(d) for d in range(2)] == ref["flags"]
    assert rep.rc == sd.SD_ERR_OVERLOAD and rep.n_hits_total == 0 == ref["n_hits"]
    assert rep.n_cand == ref["n_cand"] == [cap + 1] * 2
    assert np.array_equal(rep.zr, ref["zr"]) and np.array_equal(rep.n_hot, ref["n_hot"])
    assert rep.psi == ref["psi"]
    # every estimator is hot
    assert (ref["n_hot"] == (1 << w.k)).all()
