"""Handles used from several host threads at once (each handle by one
thread, as the header requires): every thread's windows must equal the
oracle's, whatever the interleaving of the library's calls."""
import threading

import numpy as np
import pytest

from paper_1803_11449_gb300 import traffic as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1803_11449_gb300 import build as b
    b.build()
    from paper_1803_11449_gb300 import sd as mod
    mod.lib()
    return mod


def test_threads_with_their_own_handles(sd, O):
    import torch
    w = T.WORKLOADS["tiny"].with_(dirs=2)
    wins = [T.make_window(w.with_(n=(1 << 18) + 17 * i, planted=6), 70 + i) for i in range(4)]
    out, errs = {}, []

    def run(i):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with sd.sd_create(sd.params_for(w, 700 + i, cuda_stream=s.cuda_stream)) as h:
                dev = torch.from_numpy(wins[i].pairs.reshape(-1).view(np.int32)).to("cuda", non_blocking=False)
                reps = []
                for _ in range(3):  # three windows of the same pairs, each closed and cleared
                    for part in np.array_split(np.arange(len(wins[i].pairs)), 5):
                        sd.sd_update(h, dev[2 * part[0]:2 * (part[-1] + 1)])
                    reps.append(sd.sd_close_window(h))
                out[i] = reps
        except Exception as e:  # reported below
            errs.append(e)

    ts = [threading.Thread(target=run, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    for i, win in enumerate(wins):
        op = O.params_from(w.sketch(), seed=700 + i)
        og = O.new_grid(op)
        O.update(op, og, win.pairs)
        ref = O.close_window(op, og)
        for rep in out[i]:
            assert rep.n_cand == ref["n_cand"] and np.array_equal(rep.hits["ip"], ref["ip"])
            assert np.array_equal(rep.hits["sz"], ref["sz"]) and np.array_equal(rep.hits["est"], ref["est"])
