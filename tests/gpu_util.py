"""Helpers shared by the GPU parity tests (CUDA library vs the FP64 oracle)."""
import numpy as np
import torch

import oracle as O
from paper_2007_00056_gb300 import amg


def dev():
    return torch.device("cuda", 0)


def to_cuda(sys_):
    d = dev()
    return (torch.from_numpy(sys_.rp).to(d), torch.from_numpy(sys_.ci).to(d), torch.from_numpy(sys_.val).to(d),
            torch.from_numpy(sys_.b).to(d))


def params_pair(**kw):
    """Library and oracle parameter blocks with identical settings."""
    p = amg.amg_default_params(**{k: v for k, v in kw.items() if k != "matcher"})
    okw = {k: v for k, v in kw.items() if k != "precision"}
    return p, O.Params(**okw)


def setup_both(sys_, **kw):
    p, op = params_pair(**kw)
    rp, ci, val, b = to_cuda(sys_)
    h = amg.amg_setup(rp, ci, val, p)
    oh = O.Hierarchy(sys_.rp, sys_.ci, sys_.val, params=op)
    return h, oh, b


def assert_hierarchy_bitexact(h, oh):
    """Same level count and sizes; aggregates, CSR patterns and FP64 values equal bit for bit."""
    assert h.num_levels == oh.num_levels, (h.sizes(), oh.sizes())
    for k in range(oh.num_levels):
        rp_o, ci_o, val_o, agg_o = oh.level(k)
        rp, ci, val = amg.amg_export_level(h, k)
        np.testing.assert_array_equal(rp.cpu().numpy(), rp_o, err_msg=f"row_ptr level {k}")
        np.testing.assert_array_equal(ci.cpu().numpy(), ci_o, err_msg=f"col level {k}")
        np.testing.assert_array_equal(val.cpu().numpy().view(np.int64), val_o.view(np.int64),
                                      err_msg=f"values level {k} (bitwise)")
        if agg_o is not None:
            agg = torch.empty(len(agg_o), dtype=torch.int32, device=dev())
            amg.amg_level_info(h, k, agg)
            np.testing.assert_array_equal(agg.cpu().numpy(), agg_o, err_msg=f"aggregates level {k}")


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
