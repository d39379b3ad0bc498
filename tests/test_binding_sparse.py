"""Host-side checks of the sparse binding (no GPU): CsrMatrix rejects arrays
the C ABI cannot take, before any call reaches the library."""
import numpy as np
import pytest
import torch

import synth
import paper_2002_07138_gb300 as plu


def _arrays(m=40, n=30):
    rp, ci, val = synth.sprand_csr(m, n, 0.1, seed=1)
    trp, tci, tval = synth.csr_transpose(m, n, rp, ci, val)
    return m, n, [torch.from_numpy(np.ascontiguousarray(a)) for a in (rp, ci, val, trp, tci, tval)]


def test_rejects_host_tensors():
    m, n, t = _arrays()
    with pytest.raises(ValueError):
        plu.CsrMatrix(m, n, *t)


def test_rejects_wrong_dtypes_and_sizes():
    m, n, t = _arrays()
    bad = list(t)
    bad[1] = bad[1].to(torch.int64)            # column indices must be int32
    with pytest.raises(ValueError):
        plu.CsrMatrix(m, n, *bad)
    bad = list(t)
    bad[0] = bad[0][:-1]                       # m + 1 row pointers
    with pytest.raises(ValueError):
        plu.CsrMatrix(m, n, *bad)


def test_struct_layout_matches_header():
    """The ctypes plu_csr has the header's fields in the header's order:
    three int64 then six pointers, no padding (64-bit ABI)."""
    import ctypes
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "powerlu.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} plu_csr;", hdr).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    declared = re.findall(r"(\w+)\s*[,;]", body)
    assert [f for f, _ in plu.plu_csr._fields_] == declared
    assert ctypes.sizeof(plu.plu_csr) == 3 * 8 + 6 * 8
