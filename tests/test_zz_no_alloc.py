"""The allocation-free self-energy entry point (pswf_self_energy_noalloc).

Some callers must not allocate device memory while they run -- an MD-engine
plug-in that owns every GPU buffer, or a process whose memory is all in its
own pool.  This entry point keeps its scratch in static device memory of the
library instead; the test calls it through the C-ABI twice in a row (with
different charges, so the second call reuses scratch the first one left
behind) and checks each result against pswf_self_energy on the same charges.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_self_energy_matches_existing_entry_point():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(5000, (20.0, 22.0, 18.0), (1, 2, 3, 4, 5, 6), seed=21, neutral=False)
    plan = lr.Plan(s.box, s.n, s.ps, 4.0, grid=(40, 44, 36), P=6, device=dev)
    pos = torch.tensor(s.pos, device=dev)
    rng = np.random.default_rng(5)
    for call in range(2):
        q = torch.tensor(s.q * (1.0 + call) + rng.standard_normal(s.q.shape), dtype=torch.float32, device=dev)
        plan.set_points(pos, q)
        ref = plan.self_energy()                                   # existing entry point
        out = torch.full((len(s.ps),), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        st = lr.lib().pswf_self_energy_noalloc(plan._h, s.n, ctypes.c_void_p(q.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0, lr.lib().pswf_strerror(st)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12)


def test_noalloc_rejects_bad_sizes():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan((10.0, 10.0, 10.0), 100, (1,), 3.0, grid=16, P=4, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    q = torch.zeros(1, 200, dtype=torch.float32, device=dev)
    st = lr.lib().pswf_self_energy_noalloc(plan._h, 200, ctypes.c_void_p(q.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1
