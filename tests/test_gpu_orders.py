"""Higher orders of the Fink perturbation series as MPS (Eq. 1 for n > 1,
Eq. 2): one MPS per wavefunction order, each optimised by its own sweeps, and
the Wigner 2n+1 energies E(0..2N+1) against the oracle's determinant-space
recursion (oracle.lcc.rspt, itself pinned against the direct energies
<Phi0|U|Phi(n)>).  At exact bond dimension every order is exact."""
import numpy as np
import pytest

import synth
from oracle import fci, lcc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def series():
    c = synth.config(0)
    dets = fci.determinants(8, 4, 4)
    H = fci.build_hamiltonian(c["h"], c["V"], dets)
    H0 = fci.fink_h0(H, dets, 8, c["n_core"], c["n_active"])
    E0, phi0 = fci.cas_ci(H, dets, 8, c["n_core"], c["n_active"])
    r = lcc.rspt(H, H0, phi0, 3, dets, 8, c["n_core"], c["n_active"])
    Efci, _ = fci.lowest_eigenpair(H)
    return dict(c=c, E=np.array(r["E"]), Efci=Efci)


def test_orders_one_to_three_match_the_oracle_series(mpslcc, series):
    """L=8 chain, (4e,4o) reference: M0 = 16 and M1 = 256 are exact; after
    sweeping orders 1, 2, 3 the energies E(0..7) equal the oracle's to 1e-10,
    and the third-order partial sum lies closer to full CI than the first."""
    c = series["c"]
    with mpslcc.Context(device=0, tol=1e-12) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 3)
        for n in (1, 2, 3):
            ctx.lcc_sweep(256, 3, order=n)
        E = ctx.energy_series()
        e = ctx.energy()
    ref = series["E"]
    assert len(E) == 8 and len(ref) == 8
    np.testing.assert_allclose(E, ref, atol=1e-10, rtol=0)
    assert abs(e["E2"] - ref[2]) < 1e-10 and abs(e["E3"] - ref[3]) < 1e-10
    partial = np.cumsum(E)
    assert abs(partial[7] - series["Efci"]) < abs(partial[3] - series["Efci"])


def test_order_needs_the_lower_order_and_reseeding_discards_higher(mpslcc, series):
    """Order 2 without Phi1 is a state error; re-sweeping order 1 discards
    Phi2, so the series shrinks back to E(0..3)."""
    c = series["c"]
    with mpslcc.Context(device=0, tol=1e-11) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 2)
        with pytest.raises(mpslcc.MpsLccError) as e:
            ctx.lcc_sweep(64, 1, order=2)
        assert e.value.status == 2
        ctx.lcc_sweep(256, 2, order=1)
        ctx.lcc_sweep(256, 2, order=2)
        assert len(ctx.energy_series()) == 6
        ctx.lcc_sweep(256, 1, order=1)
        assert len(ctx.energy_series()) == 4
