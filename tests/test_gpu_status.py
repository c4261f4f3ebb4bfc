"""Device-side status through the C ABI: pt_domain_check counts parameter
sets outside the model's domain, and pt_status_read turns that count, or a
Newton non-convergence count, into PT_ERR_DOMAIN / PT_ERR_NOT_CONVERGED.

The out-of-domain parameters go only to pt_domain_check, which reads them;
no light-curve kernel is run on them.  Non-convergence is made with a valid
eccentric workload and a step cap of one Newton step (every loop is bounded).
"""
import numpy as np
import pytest

from paper_1504_07433_gb300 import workloads as W
from tests.helpers import gpu_inputs

pytestmark = pytest.mark.gpu

PT_OK, PT_ERR_DOMAIN, PT_ERR_NOT_CONVERGED = 0, 2, 3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    pt.load_library()
    return torch


def test_domain_check_counts_bad_parameter_sets(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=64, n_t=10)
    t, orb, k, ld = gpu_inputs(wl)
    n = pt.domain_check(orb, k)
    assert int(n.item()) == 0
    assert pt.status_read(None, n) == (PT_OK, "")
    # plant one fault per chosen vector, each in a different parameter
    kb = k.clone()
    o = {kk: (None if vv is None else vv.clone()) for kk, vv in orb.items()}
    kb[3] = 0.0
    kb[5] = float("nan")
    kb[7] = -0.1
    o["a"][11] = 0.9
    o["e"][13] = 0.97
    o["P"][17] = 0.0
    o["inc"][19] = -0.2
    o["w"][23] = float("inf")
    o["t0"][29] = float("nan")
    n = pt.domain_check(o, kb)
    assert int(n.item()) == 9
    st, msg = pt.status_read(None, n)
    assert st == PT_ERR_DOMAIN and "9" in msg
    # per-passband radius ratios: every bad ratio counts
    kp = torch.stack([k, k, k], dim=1).contiguous()
    kp[2, 1] = 0.0
    kp[2, 2] = 0.0
    kp[40, 0] = float("nan")
    assert int(pt.domain_check(orb, kp).item()) == 3
    # a circular orbit has no e, w to check
    oc = dict(orb, e=None, w=None)
    assert int(pt.domain_check(oc, k).item()) == 0


def test_newton_step_cap_reported_as_not_converged(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=32, n_t=3000, n_ss=4, cadence=0.011)
    t, orb, k, ld = gpu_inputs(wl)
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    pt.ma_quad(t, orb, k, ld, n_ss=4, t_exp=wl["t_exp"], max_iter=16, n_bad=bad)
    assert pt.status_read(bad, None) == (PT_OK, "")
    pt.ma_quad(t, orb, k, ld, n_ss=4, t_exp=wl["t_exp"], max_iter=1, n_bad=bad)
    st, msg = pt.status_read(bad, None)
    assert st == PT_ERR_NOT_CONVERGED and int(bad.item()) > 0
    # a domain fault outranks non-convergence
    nd = torch.ones(1, dtype=torch.int32, device="cuda")
    assert pt.status_read(bad, nd)[0] == PT_ERR_DOMAIN
    # the FP64 Newton of pt_z_ecc reports through the same counter
    z, nb = pt.z_ecc(t, orb, n_ss=1, max_iter=1, tol=1e-14)
    assert pt.status_read(nb, None)[0] == PT_ERR_NOT_CONVERGED
