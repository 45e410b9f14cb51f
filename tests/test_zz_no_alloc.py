"""The allocation-free D_W entry point (smpq_dslash_noalloc) against smpq_dslash.

smpq_dslash_noalloc serves callers that cannot allocate device memory (their
memory belongs to another allocator, or cudaMalloc's device synchronisation is
not acceptable where they call from).  It keeps its scratch in a fixed 32 MiB
device array, so this test checks that two calls in a row, with different
inputs and options, each reproduce smpq_dslash, and that a field too large for
the scratch is rejected.  The file sorts last so that a run stopping at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

from synth import make_config, random_spinor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_and_torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02211_gb300 import Session
    cfg = make_config("flux4x8")
    s = Session(device=0)
    s.load_gauge(cfg["dims"], cfg["U"])
    yield s, torch, int(np.prod(cfg["dims"]))
    s.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
def test_noalloc_matches_dslash_twice(ctx_and_torch, precision, tol):
    from paper_1901_02211_gb300 import smpq
    s, torch, V = ctx_and_torch
    rng = np.random.default_rng(17)
    for call, (B, dagger) in enumerate([(3, False), (2, True)]):  # two calls in a row, different inputs
        psi = _dev(torch, random_spinor(rng, V, B))
        ref = torch.empty_like(psi)
        got = torch.full_like(psi, float("nan"))
        smpq.smpq_dslash(s.ctx, psi, ref, B, dagger, precision)
        smpq.smpq_dslash_noalloc(s.ctx, psi, got, B, dagger, precision)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item()
        scale = ref.abs().max().item() if precision == 1 else 1.0
        assert err <= tol * scale, "call %d: max |diff| = %g" % (call, err)


def test_noalloc_rejects_fields_beyond_the_scratch(ctx_and_torch):
    from paper_1901_02211_gb300 import smpq
    s, torch, V = ctx_and_torch
    B = (32 << 20) // (2 * V * 12 * 16) + 1  # one column more than the FP64 limit
    psi = torch.zeros((V, 4, 3, B), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    with pytest.raises(smpq.SmpqError) as e:
        smpq.smpq_dslash_noalloc(s.ctx, psi, out, B, False, smpq.SMPQ_FP64)
    assert e.value.code == smpq.SMPQ_EINVAL
    assert "32" in str(e.value) or "limit" in str(e.value)
