"""The C ABI library builds, loads without a GPU, exports every declared symbol,
and its host-side logic (Zolotarev coefficients, colouring, validation) agrees
with the oracle.  No GPU compute is called here."""
import os
import re

import numpy as np
import pytest

from oracle import probing, zolotarev
from paper_1901_02211_gb300 import smpq as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "smpq.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(smpq_[a-z_0-9]+)\s*\(", txt)))


def test_library_loads_and_exports_every_declared_symbol():
    L = S.load()
    decl = _declared()
    assert len(decl) >= 16
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(S.EXPORTS)


def test_options_default_are_the_papers():
    o = S.smpq_options_default()
    assert o.kappa == 0.21 and o.npoles == 14  # Sec. 2.1
    assert o.tol == 1e-10 and list(o.bc) == [1, 1, 1, 1]


@pytest.mark.parametrize("n,a,b", [(14, 0.0193, 7.0), (14, 1e-3, 8.0), (6, 0.1, 7.0), (20, 1e-4, 10.0)])
def test_zolotarev_matches_oracle(n, a, b):
    c0, c, q, d = S.smpq_zolotarev(n, a, b)
    r0, rc, rq, rd = zolotarev.zolotarev(n, a, b)
    assert abs(c0 - r0) <= 1e-12 * r0
    assert np.allclose(c, rc, rtol=1e-11, atol=0)
    assert np.allclose(q, rq, rtol=1e-11, atol=0)
    assert abs(d - rd) <= 1e-13  # delta is a difference of two O(1) numbers


def test_zolotarev_rejects_bad_interval():
    with pytest.raises(S.SmpqError):
        S.smpq_zolotarev(14, 0.0, 1.0)
    with pytest.raises(S.SmpqError):
        S.smpq_zolotarev(14, 2.0, 1.0)
    with pytest.raises(S.SmpqError):
        S.smpq_zolotarev(33, 0.1, 1.0)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 16), (12, 12, 12, 24)])
@pytest.mark.parametrize("r,mode", [(2, 0), (4, 0), (2, 1), (2, 2), (4, 2), (4, 1), (3, 0)])
def test_colouring_matches_oracle(dims, r, mode):
    try:
        ref, nref = probing.color_sites(dims, r, mode)
    except ValueError:
        with pytest.raises(S.SmpqError) as e:
            S.smpq_colour_sites(dims, r, mode)
        assert e.value.code == S.SMPQ_EINVAL
        return
    col, n = S.smpq_colour_sites(dims, r, mode)
    assert n == nref
    assert np.array_equal(col, ref)


def test_colouring_point_sources():
    dims = (4, 4, 4, 8)
    col, n = S.smpq_colour_sites(dims, 4, 0)
    assert n == 256
    with pytest.raises(S.SmpqError):
        S.smpq_colour_sites(dims, 8, 0)  # 8 does not divide 4


def test_binding_constants_match_the_header():
    """Every enumerator of include/smpq.h (status codes, precisions) has the same
    value in the Python binding."""
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(SMPQ_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt))
    assert {"SMPQ_FP64", "SMPQ_FP32", "SMPQ_MIXED", "SMPQ_FP16N", "SMPQ_BF16N", "SMPQ_OK", "SMPQ_EINVAL"} <= set(enums)
    for name, value in enums.items():
        assert getattr(S, name) == value, name


def _struct_members(name):
    """Member names of `typedef struct { ... } name;` in include/smpq.h, in order."""
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", txt).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            out.extend(re.sub(r"\[.*?\]", "", v).split()[-1].lstrip("*") for v in decl.split(","))
    return out


@pytest.mark.parametrize("cname,pyclass", [("smpq_options", S.smpq_options), ("smpq_stats", S.smpq_stats)])
def test_binding_structs_follow_the_header(cname, pyclass):
    """The ctypes mirrors of the option and statistics structs have the header's
    members in the header's order (a drift would shift every later field)."""
    assert [f for f, _ in pyclass._fields_] == _struct_members(cname)


def test_buffer_checks_refuse_before_any_launch(monkeypatch):
    """The binding refuses a buffer of the wrong type or size before calling C
    (a short or complex64 buffer would be overrun by the kernels).  The
    context's lattice comes from a stand-in for smpq_context_info (no GPU here)."""
    monkeypatch.setattr(S, "smpq_context_info", lambda ctx: ((4, 4, 4, 4), 0))
    V, B = 256, 3
    good = np.zeros((V, 4, 3, B), dtype=np.complex128)
    S._check_fields(None, good, good, B)  # accepted
    with pytest.raises(ValueError, match="dtype"):
        S._check_fields(None, good.astype(np.complex64), good, B)
    with pytest.raises(ValueError, match="elements"):
        S._check_fields(None, good, good[:, :, :, :2].copy(), B)
    S._check_sites(None, np.zeros(V), np.zeros(V), ("q_re", "q_im"))
    with pytest.raises(ValueError, match="elements"):
        S._check_sites(None, np.zeros(V - 1), np.zeros(V), ("q_re", "q_im"))
    with pytest.raises(ValueError, match="dtype"):
        S._check_sites(None, np.zeros(V, dtype=np.float32), np.zeros(V), ("q_re", "q_im"))
    monkeypatch.setattr(S, "smpq_context_info", lambda ctx: ((0, 0, 0, 0), 0))
    with pytest.raises(S.SmpqError):
        S._volume(None)


def test_tune_cache_round_trip(tmp_path):
    """The autotuner's cache file: a stored shape is found again for the same
    key only, the last matching line wins, malformed lines are skipped and a
    missing file reads as 'not found' (host code, no GPU)."""
    path = str(tmp_path / "tune.txt")
    dev, dims = "NVIDIA GB300/152sm", (8, 8, 8, 16)
    assert S.smpq_tune_cache_lookup(path, dev, dims, 3072, S.SMPQ_MIXED) is None
    S.smpq_tune_cache_store(path, dev, dims, 3072, S.SMPQ_MIXED, (48, 4, 2, 1, 1), 7.5)
    S.smpq_tune_cache_store(path, dev, dims, 1536, S.SMPQ_MIXED, (24, 1, 8, 2, 0), 3.0)
    assert S.smpq_tune_cache_lookup(path, dev, dims, 3072, S.SMPQ_MIXED) == (48, 4, 2, 1, 1)
    assert S.smpq_tune_cache_lookup(path, dev, dims, 1536, S.SMPQ_MIXED) == (24, 1, 8, 2, 0)
    assert S.smpq_tune_cache_lookup(path, dev, dims, 3072, S.SMPQ_FP32) is None
    assert S.smpq_tune_cache_lookup(path, dev, (8, 8, 16, 8), 3072, S.SMPQ_MIXED) is None
    assert S.smpq_tune_cache_lookup(path, "other/1sm", dims, 3072, S.SMPQ_MIXED) is None
    with open(path, "a") as f:
        f.write("smpq-tune-2|NVIDIA GB300/152sm|8 8 8 16|3072|2|7 4 4 1 0|1.0\n")  # tile 7: rejected
        f.write("smpq-tune-2|NVIDIA GB300/152sm|8 8 8 16|3072|2|48 4 4 2 1|1.0\n")  # staged needs nr 1
        f.write("smpq-tune-1|NVIDIA GB300/152sm|8 8 8 16|3072|2|48 8 8 1|1.0\n")  # old format: ignored
        f.write("garbage line\n")
    assert S.smpq_tune_cache_lookup(path, dev, dims, 3072, S.SMPQ_MIXED) == (48, 4, 2, 1, 1)
    S.smpq_tune_cache_store(path, dev, dims, 3072, S.SMPQ_MIXED, (12, 8, 8, 2, 0), 6.0)
    assert S.smpq_tune_cache_lookup(path, dev, dims, 3072, S.SMPQ_MIXED) == (12, 8, 8, 2, 0)
    with pytest.raises(S.SmpqError):
        S.smpq_tune_cache_store(path, "bad|name", dims, 3072, S.SMPQ_MIXED, (48, 4, 4, 1, 0), 1.0)
