"""GPU energies of finite-bond-dimension states against the oracle.

At a bond dimension below the exact one the sweeps truncate (discarded weight
> 0), so the first-order MPS is neither the exact Fink first-order state nor
exactly orthogonal to the reference.  The library reports the energies OF ITS
STATES (Eq. 1b for E2 = J(Q Phi1), Eq. 2 with n = 1 for E3); the oracle
evaluates the same definitions on the exported states expanded into
determinants (Eq. mps1), so the two must agree to 1e-10 at any bond
dimension, whatever precision steered the optimisation."""
import numpy as np
import pytest

import synth
from oracle import fci, lcc, mps as omps

pytestmark = pytest.mark.gpu

ENERGY_TOL = 1e-10


@pytest.fixture(scope="module")
def chain():
    c = synth.config(0)
    dets = fci.determinants(8, 4, 4)
    H = fci.build_hamiltonian(c["h"], c["V"], dets)
    H0 = fci.fink_h0(H, dets, 8, c["n_core"], c["n_active"])
    exact = lcc.lcc_energies(c["h"], c["V"], 4, 4, c["n_core"], c["n_active"])
    return dict(c=c, dets=dets, H=H, H0=H0, exact=exact)


def mps_sum(a, b, cb):
    """MPS of Phi_a + cb * Phi_b by the direct sum of the interior bond spaces
    (block-diagonal interior site tensors; the first site concatenates along
    its right bond, the last stacks along its left bond)."""
    k = len(a["sites"])
    bonds, offs = [], []
    for bnd in range(k + 1):
        qa = {(n, s): d for (n, s, d) in a["bonds"][bnd]}
        qb = {(n, s): d for (n, s, d) in b["bonds"][bnd]}
        keys = sorted(set(qa) | set(qb))
        if bnd in (0, k):
            assert qa == qb and len(keys) == 1
            bonds.append([(keys[0][0], keys[0][1], 1)])
            offs.append({keys[0]: (0, 0, 0)})
            continue
        bonds.append([(q[0], q[1], qa.get(q, 0) + qb.get(q, 0)) for q in keys])
        offs.append({q: (i, 0, qa.get(q, 0)) for i, q in enumerate(keys)})
    sites = []
    for p in range(k):
        blocks = {}
        for src, scale, part in ((a, 1.0, 1), (b, cb if p == 0 else 1.0, 2)):
            for (ia, s, ib), blk in src["sites"][p].items():
                qL = tuple(src["bonds"][p][ia][:2])
                qR = tuple(src["bonds"][p + 1][ib][:2])
                IL, oL = offs[p][qL][0], offs[p][qL][part]
                IR, oR = offs[p + 1][qR][0], offs[p + 1][qR][part]
                key = (IL, s, IR)
                if key not in blocks:
                    blocks[key] = np.zeros((bonds[p][IL][2], bonds[p + 1][IR][2]))
                blocks[key][oL:oL + blk.shape[0], oR:oR + blk.shape[1]] += scale * blk
        sites.append(blocks)
    masks = [tuple(sorted({key[1] for key in s})) for s in sites]
    return dict(bonds=bonds, sites=sites, masks=masks)


def _check_states(ctx, ch, e):
    p0, p1 = ctx.export_mps(0), ctx.export_mps(1)
    v0 = omps.to_vector(p0, ch["dets"])
    v1 = omps.to_vector(p1, ch["dets"])
    o = lcc.state_energies(ch["H"], ch["H0"], v0, v1)
    assert abs(np.linalg.norm(v0) - 1.0) < 1e-10
    assert abs(e["E0"] - o["E0"]) <= ENERGY_TOL, (e["E0"], o["E0"])
    assert abs(e["E2"] - o["E2"]) <= ENERGY_TOL, (e["E2"], o["E2"])
    assert abs(e["E3"] - o["E3"]) <= ENERGY_TOL, (e["E3"], o["E3"])
    assert abs(e["overlap01"] - o["overlap01"]) <= 1e-10
    assert abs(e["norm1"] - o["norm1"]) <= 1e-10 * max(1.0, o["norm1"])
    return o


@pytest.mark.parametrize("prec", ["FP64", "BF16X3"])
def test_config1_truncated_states_match_oracle(mpslcc, chain, prec):
    """The L=8 chain as configured: reference M0 = 16 (exact), first order
    M1 = 64 (the middle bond's exact dimension is 256), 4 sweeps.  Truncation
    discards weight; the energies of the resulting states equal the oracle's
    evaluation of the exported states; the Hylleraas value lies above the exact
    E2 (A is positive definite on the Q space here) and below zero."""
    c = chain["c"]
    kw = dict(refine_steps=12) if prec != "FP64" else {}
    with mpslcc.Context(device=0, prec=getattr(mpslcc, prec), tol=1e-10, **kw) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(c["M0"], c["sweeps"])
        ctx.lcc_sweep(c["M1"], c["sweeps"])
        e = ctx.energy()
        o = _check_states(ctx, chain, e)
        disc = e["max_discarded_weight"]
    ex = chain["exact"]
    assert disc > 1e-8, disc
    assert ex["E2"] - 1e-10 <= o["E2"] < 0.0
    assert o["E2"] - ex["E2"] < 0.05 * abs(ex["E2"])


def test_loaded_states_with_reference_admixture(mpslcc, chain):
    """Energies of loaded states whose first-order MPS overlaps the reference
    (Phi1 = a random MPS + c Phi0, so s = <Phi1|Phi0> is about c = 0.5 or
    -0.25): the s-dependent terms of the FP64 energy passes are exercised
    directly.  Loading Phi0 itself as Phi1 (s = 1, so
    Q Phi1 = 0) gives J = E3 = 0."""
    c = chain["c"]
    with mpslcc.Context(device=0, tol=1e-11) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 3)
        p0 = ctx.export_mps(0)
        for seed, cb in ((3, 0.5), (4, -0.25)):
            phi1 = mps_sum(synth.random_mps(8, 8, 0, M=48, seed=seed, isometric=False), p0, cb)
            ctx.load_mps(1, phi1)
            e = ctx.energy()
            o = _check_states(ctx, chain, e)
            assert abs(o["overlap01"] - cb) < 0.05, o["overlap01"]
        ctx.load_mps(1, p0)
        e = ctx.energy()
        o = _check_states(ctx, chain, e)
    assert abs(o["overlap01"] - 1.0) < 1e-10
    assert abs(e["E2"]) < 1e-10 and abs(e["E3"]) < 1e-10


@pytest.mark.parametrize("prec", ["FP64", "BF16X3"])
def test_sweep_windows_reproduce_the_sweep_bit_for_bit(mpslcc, chain, prec):
    """A full sweep run as two windows (positions 0..6 left to right, then
    6..0 right to left) gives the same states and energies as mpslcc_lcc_sweep,
    to the last bit: the split-K partial sums are added in a fixed order, so
    two runs of the same work agree exactly."""
    c = chain["c"]
    res = []
    for mode in ("sweep", "windows", "sweep"):
        with mpslcc.Context(device=0, prec=getattr(mpslcc, prec), tol=1e-10) as ctx:
            ctx.build_mpo(c["h"], c["V"], 8, 0)
            ctx.set_spaces(c["n_core"], c["n_active"])
            ctx.dmrg_reference(16, 2)
            ctx.lcc_sweep(64, 1)
            if mode == "sweep":
                ctx.lcc_sweep(64, 1)
            else:
                ctx.lcc_window(64, 0, 7, 1)
                ctx.lcc_window(64, 6, 7, -1)
            e = ctx.energy()
            p1 = ctx.export_mps(1)
        res.append((e, np.concatenate([b.ravel() for s in p1["sites"] for _, b in sorted(s.items())])))
    for e, v in res[1:]:
        for key in ("E0", "E2", "E3"):
            assert e[key] == res[0][0][key], (key, e[key], res[0][0][key])
        assert np.array_equal(v, res[0][1])
