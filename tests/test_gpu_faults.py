"""Failure detection without a GPU fault: every failure below is made on the
host (an allocator that refuses, an iteration cap) or by a device wait whose
bound runs out on valid work, and each call must return its status while the
context stays usable."""
import json
import os
import warnings

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_energies.json")))


def _bf16(x):
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_wait_bound_expiry_returns_timeout(mpslcc):
    """A one-microsecond bound on the tensor-core kernel's mbarrier waits runs
    out on a long product: the kernel records the expiry, waits for the loads
    and products it already issued, frees its tensor memory and returns; the
    call reports E_TIMEOUT, again on a second call, and the GPU and a context
    with the default bound still compute the product correctly."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((512, 8192))
    B = rng.standard_normal((384, 8192))
    ref = _bf16(A) @ _bf16(B).T
    with mpslcc.Context(device=0, wait_timeout_s=1e-6) as ctx:
        for _ in range(2):
            with pytest.raises(mpslcc.MpsLccError) as e:
                ctx.debug_tc_gemm(A, B, prec=mpslcc.BF16, mode=2)
            assert e.value.status == 6, str(e.value)
        # the context stays usable for work that needs no tensor-core wait
        c = synth.config(0)
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        E0 = ctx.dmrg_reference(16, 2)
        assert abs(E0 - GOLDEN["hubbard1d_L8_U4"]["E0"]) < 1e-8
    with mpslcc.Context(device=0) as ctx:
        C = ctx.debug_tc_gemm(A, B, prec=mpslcc.BF16, mode=2)
    assert np.abs(C - ref).max() / np.abs(ref).max() < 1e-5


class _FlakyAllocator:
    """Device allocator over PyTorch's caching allocator that refuses its
    N-th request, as an exhausted pool would: it returns NULL, or raises (as
    PyTorch's own allocator does when it runs out of memory)."""

    def __init__(self, torch, stream, raise_on_failure=False):
        self.torch, self.stream = torch, stream
        self.count, self.fail_at, self.live = 0, None, {}
        self.raise_on_failure = raise_on_failure

    def alloc(self, nbytes):
        self.count += 1
        if self.fail_at is not None and self.count == self.fail_at:
            if self.raise_on_failure:
                raise MemoryError("refused by the test allocator")
            return 0
        p = self.torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), 0, self.stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes):
        if ptr in self.live:
            del self.live[ptr]
            self.torch.cuda.caching_allocator_delete(ptr)


@pytest.mark.parametrize("raise_on_failure", [False, True])
def test_failed_allocation_returns_nomem_and_context_recovers(mpslcc, raise_on_failure):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(0)
    fa = _FlakyAllocator(torch, stream, raise_on_failure)
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-11, alloc=(fa.alloc, fa.free), stream=stream.cuda_stream) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        fa.fail_at = fa.count + 200   # an allocation in the middle of the reference sweeps
        with pytest.raises(mpslcc.MpsLccError) as e:
            ctx.dmrg_reference(16, 3)
        assert e.value.status == 4, str(e.value)
        assert fa.count >= fa.fail_at
        fa.fail_at = None
        E0 = ctx.dmrg_reference(16, 3)
        assert abs(E0 - GOLDEN["hubbard1d_L8_U4"]["E0"]) < 1e-10
        ctx.lcc_sweep(256, 2)
        e2 = ctx.energy()
    torch.cuda.synchronize()
    assert not fa.live, "every device allocation was returned"
    assert abs(e2["E2"] - GOLDEN["hubbard1d_L8_U4"]["E2"]) < 1e-10


def test_iteration_cap_returns_noconv_with_results_kept(mpslcc):
    """max_iter = 1: the local solves stop early, the calls complete, report
    E_NOCONV (a warning in the binding) and keep finite states and energies."""
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-12, max_iter=1) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        with pytest.warns(mpslcc.MpsLccNoConvergence):
            E0 = ctx.dmrg_reference(16, 1)
        assert ctx.last_status == mpslcc.E_NOCONV and np.isfinite(E0)
        with pytest.warns(mpslcc.MpsLccNoConvergence):
            E2 = ctx.lcc_sweep(64, 1)
        assert ctx.last_status == mpslcc.E_NOCONV and np.isfinite(E2)
        e = ctx.energy()
        st = ctx.stats()
    assert e["flags"] & mpslcc.FLAG_NOCONV
    assert st["n_noconv"] > 0
    assert np.isfinite(e["E2"]) and np.isfinite(e["E3"])


def test_poor_reference_is_flagged(mpslcc):
    """A one-determinant reference (M0 = 1) is not the lowest H0 state of the
    reference class, so Q(H0 - E0)Q is indefinite and the Hylleraas
    functional has no minimum: the local solves meet non-positive curvature
    and the energies carry the flag."""
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-10, init_guess=1) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(1, 1)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", mpslcc.MpsLccNoConvergence)
            ctx.lcc_sweep(64, 1)
        e = ctx.energy()
        st = ctx.stats()
    assert e["flags"] & mpslcc.FLAG_INDEFINITE, e["flags"]
    assert st["n_indefinite"] > 0
