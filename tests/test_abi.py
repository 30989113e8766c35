"""CPU checks of the C ABI: the library loads, exports every entry point that
include/qem.h declares, and rejects invalid descriptors on the host before
touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2503_08264_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qem_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_08264_gb300 import build
    build.build()
    return L.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.SIGNATURES), "binding signatures must mirror the header"


def test_status_strings(lib):
    for code in range(7):
        assert lib.qem_status_string(code).startswith(b"QEM_")


def _desc(levels):
    d = L.ModelDesc()
    d.n_levels = len(levels)
    keep = []
    for i, kw in enumerate(levels[:L.QEM_MAX_LEVELS]):
        lv = d.levels[i]
        for k, v in kw.items():
            if k == "parent" and v is not None:
                arr = np.ascontiguousarray(v, np.int64)
                keep.append(arr)
                v = arr.ctypes.data
            setattr(lv, k, v)
    return d, keep


ROOT_LV = dict(n=1, dim=2, prior=0, prior_a=1.0, qfam=0)


def _child(**kw):
    base = dict(n=3, dim=2, prior=1, prior_a=1.0, qfam=0, parent=[0, 0, 0])
    base.update(kw)
    return base


@pytest.mark.parametrize("levels,K", [
    ([], 8),                                                   # no level
    ([ROOT_LV] * 5, 8),                                        # too many levels
    ([ROOT_LV, _child()], 0),                                  # K = 0
    ([ROOT_LV, _child()], 5000),                               # K too large
    ([ROOT_LV, _child(parent=[0, 1, 0])], 8),                  # parent out of range
    ([dict(ROOT_LV, n=2), _child(parent=[1, 0, 1])], 8),       # parents not grouped
    ([ROOT_LV, _child(dim=3)], 8),                             # fixed-var prior, dim mismatch
    ([ROOT_LV, _child(prior=2)], 8),                           # mean/log-var prior needs parent dim 2D
    ([ROOT_LV, _child(lik=2, n_obs=4)], 8),                    # likelihood without data pointers
    ([ROOT_LV, _child(parent=None)], 8),                       # missing parents
    ([dict(ROOT_LV, prior=1)], 8),                             # root with a parent-relative prior
    ([dict(ROOT_LV, n=-1)], 8),                                # negative size
    ([ROOT_LV, _child(n=4, parent=[0] * 4, chain=3, prior_b=0.1)], 8),          # days not whole chains
    ([ROOT_LV, _child(n=4, parent=[0] * 4, chain=2)], 8),                        # chain without a step variance
    ([dict(ROOT_LV, n=2), _child(n=4, parent=[0, 0, 0, 1], chain=2, prior_b=0.1)], 8),  # parent changes in a chain
    ([ROOT_LV, _child(chain=-1)], 8),                          # negative chain length
])
def test_invalid_descriptors_rejected_on_host(lib, levels, K):
    d, keep = _desc(levels)
    o = L.PlanOpts()
    o.K = K
    h = C.c_void_p()
    rc = lib.qem_plan(C.byref(d), C.byref(o), C.byref(h))
    assert rc == L.QEM_ERR_INVALID_ARG
    assert not h.value


@pytest.mark.parametrize("levels", [
    [dict(ROOT_LV, dim=65)],                                                            # dimension too large
    [dict(ROOT_LV, dim=1, qfam=1, prior=3, prior_a=2.0, prior_b=1.0), _child(dim=1)],  # Gamma q inside a tree
    [dict(ROOT_LV, chain=2)],                                                           # chain at the root
    [ROOT_LV, _child(n=4, parent=[0] * 4, chain=2, prior_b=0.1), _child(n=1, parent=[0])],  # chain not the leaf
    [dict(ROOT_LV, dim=9), _child(n=4, dim=9, parent=[0] * 4, chain=2, prior_b=0.1)],   # chain dimension above 8
])
def test_unsupported_requests(lib, levels):
    d, keep = _desc(levels)
    o = L.PlanOpts()
    o.K = 8
    h = C.c_void_p()
    assert lib.qem_plan(C.byref(d), C.byref(o), C.byref(h)) == L.QEM_ERR_UNSUPPORTED


def test_null_arguments(lib):
    assert lib.qem_plan(None, None, None) == L.QEM_ERR_INVALID_ARG
    assert lib.qem_estep(None, None, None, 0, 0, None, None) == L.QEM_ERR_INVALID_ARG
    assert lib.qem_mstep(None, None, None, None, 0.5, 0.0, 1) == L.QEM_ERR_INVALID_ARG
    assert lib.qem_plan_destroy(None) == L.QEM_OK


def test_chain_plans_need_the_fp32_path(lib):
    d, keep = _desc([ROOT_LV, _child(n=4, parent=[0] * 4, chain=2, prior_b=0.1)])
    o = L.PlanOpts()
    o.K = 128
    o.precision = L.QEM_PREC_BF16X3
    h = C.c_void_p()
    assert lib.qem_plan(C.byref(d), C.byref(o), C.byref(h)) == L.QEM_ERR_UNSUPPORTED
    o.precision = L.QEM_PREC_FP32
    o.K = 2048
    assert lib.qem_plan(C.byref(d), C.byref(o), C.byref(h)) == L.QEM_ERR_UNSUPPORTED
