"""The binding of rts_bin_noalloc checks its arguments before any pointer reaches the
library (which writes n entries of key and perm and nblocks + 1 of cstart into device
memory): host arrays, wrong dtypes or shapes and short buffers raise ValueError.  No GPU
is needed: every case is rejected before the library is called."""
import numpy as np
import pytest
import torch

from paper_2009_14514_gb300 import rts, scenes


def _args(n=10, nb=None, **over):
    sc = scenes.wcsph_dam_break_8k()
    P = rts.make_params(sc.params)
    nblocks = int(np.prod(sc.params["grid_dim"]))
    a = dict(x=torch.zeros((n, 3), dtype=torch.float32), key=torch.zeros(n, dtype=torch.int32),
             perm=torch.zeros(n, dtype=torch.int32),
             cstart=torch.zeros(nblocks + 1 if nb is None else nb, dtype=torch.int32))
    a.update(over)
    return P, a


@pytest.mark.parametrize("case, msg", [
    ("numpy_x", "torch tensor"),
    ("x_float64", "float32 of shape"),
    ("x_shape", "float32 of shape"),
    ("key_int64", "key must be int32"),
    ("perm_short", "perm holds"),
    ("cstart_short", "cstart holds"),
    ("host_tensors", "device memory"),
    ("non_contiguous", "contiguous"),
])
def test_noalloc_binding_rejects_bad_arguments(case, msg):
    n = 10
    if case == "numpy_x":
        P, a = _args(x=np.zeros((n, 3), np.float32))
    elif case == "x_float64":
        P, a = _args(x=torch.zeros((n, 3), dtype=torch.float64))
    elif case == "x_shape":
        P, a = _args(x=torch.zeros((n, 4), dtype=torch.float32))
    elif case == "key_int64":
        P, a = _args(key=torch.zeros(n, dtype=torch.int64))
    elif case == "perm_short":
        P, a = _args(perm=torch.zeros(n - 1, dtype=torch.int32))
    elif case == "cstart_short":
        P, a = _args(nb=100)
    elif case == "host_tensors":
        P, a = _args()
    else:
        P, a = _args(x=torch.zeros((3, n), dtype=torch.float32).t())
    with pytest.raises(ValueError, match=msg):
        rts.rts_bin_noalloc(P, a["x"], a["key"], a["perm"], a["cstart"])
