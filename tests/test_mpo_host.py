"""Host-side checks of the C-ABI library (no GPU): exported symbols and the
MPO builder, contracted densely and compared with the oracle's
determinant-space Hamiltonian over the whole Fock space."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import fci

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol(mpslcc):
    hdr = open(os.path.join(ROOT, "include", "mpslcc.h")).read()
    names = set(re.findall(r"\b(mpslcc_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 18
    lib = ctypes.CDLL(mpslcc.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(mpslcc.EXPORTED) <= names


def _dense_mpo(ctx, which, k):
    dims = ctx.mpo_bond_dims(which)
    T = np.ones((1, 1, 1))  # [w, S', S]
    for p in range(k):
        idx, val = ctx.export_mpo_site(which, p)
        W = np.zeros((dims[p], dims[p + 1], 4, 4))
        for (w0, w1, so, si), v in zip(idx, val):
            W[w0, w1, so, si] += v
        T = np.einsum("wab,wvcd->vacbd", T, W).reshape(dims[p + 1], T.shape[1] * 4, T.shape[2] * 4)
    assert T.shape[0] == 1
    return T[0]


def _fock_dets(k):
    return np.arange(4 ** k, dtype=np.int64)  # every bit mask (sorted)


def _site_index(D, k):
    S = 0
    for p in range(k):
        s = ((D >> (2 * p)) & 1) + 2 * ((D >> (2 * p + 1)) & 1)
        S = S * 4 + s
    return S


def _integrals(k, seed):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((k, k))
    h = 0.5 * (h + h.T)
    V = np.zeros((k,) * 4)
    for _ in range(2):
        B = rng.standard_normal((k, k)) * 0.4
        B = 0.5 * (B + B.T)
        V += np.einsum("ij,kl->ijkl", B, B)
    return h, V


@pytest.mark.parametrize("k,nc,na", [(2, 0, 2), (3, 1, 1), (4, 1, 2), (5, 1, 2)])
def test_mpo_equals_fock_hamiltonian(mpslcc, k, nc, na):
    h, V = _integrals(k, 100 + k)
    ctx = mpslcc.Context(device=-1)
    ctx.build_mpo(h, V, n_elec=k, two_sz=k % 2)
    ctx.set_spaces(nc, na)
    dets = _fock_dets(k)
    perm = np.array([_site_index(int(D), k) for D in dets])
    Hf = fci.build_hamiltonian(h, V, dets).toarray()
    H0f = fci.build_hamiltonian(h, V, dets, fci.delta_nex_zero(k, nc, na)).toarray()
    for which, ref in ((mpslcc.MPO_H, Hf), (mpslcc.MPO_H0, H0f), (mpslcc.MPO_U, Hf - H0f)):
        M = _dense_mpo(ctx, which, k)
        R = np.zeros_like(M)
        R[np.ix_(perm, perm)] = ref
        np.testing.assert_allclose(M, R, atol=1e-12, rtol=0, err_msg=f"MPO kind {which}")
    Mi = _dense_mpo(ctx, mpslcc.MPO_ID, k)
    np.testing.assert_allclose(Mi, np.eye(4 ** k), atol=0)
    ctx.close()


def test_mpo_bond_dimension_bound(mpslcc):
    """D <= 2 + 4k + 8 min(n_left, n_right)^2 (channels labelled by at most
    two operators; Implementation section: O(k^2))."""
    c = synth.config(1)
    ctx = mpslcc.Context(device=-1)
    ctx.build_mpo(c["h"], c["V"], 24, 0)
    dims = ctx.mpo_bond_dims(mpslcc.MPO_H)
    k = 24
    for b in range(k + 1):
        m = min(b, k - b)
        assert dims[b] <= 2 + 4 * k + 8 * m * m, (b, dims[b])
    assert dims[0] == 1 and dims[k] == 1
    ctx.close()


def test_build_mpo_rejects_bad_input(mpslcc):
    h, V = _integrals(3, 1)
    ctx = mpslcc.Context(device=-1)
    with pytest.raises(mpslcc.MpsLccError) as e:
        ctx.build_mpo(h, V, n_elec=3, two_sz=0)  # parity
    assert e.value.status == 1
    hb = h.copy()
    hb[0, 1] += 1.0
    with pytest.raises(mpslcc.MpsLccError):
        ctx.build_mpo(hb, V, n_elec=2, two_sz=0)
    with pytest.raises(mpslcc.MpsLccError) as e:
        ctx.set_spaces(1, 1)  # before build_mpo
    assert e.value.status == 2
    ctx.close()


def test_host_only_context_contract(mpslcc):
    """Option checks run at creation; a host-only context (device = -1) builds
    and exports MPOs but refuses every call that runs kernels, with E_STATE and
    a message, and stays usable afterwards."""
    for kw in ({"prec": 7}, {"init_guess": 3}):
        with pytest.raises(mpslcc.MpsLccError) as e:
            mpslcc.Context(device=-1, **kw)
        assert e.value.status == 1
    h, V = _integrals(4, 2)
    ctx = mpslcc.Context(device=-1)
    ctx.build_mpo(h, V, n_elec=4, two_sz=0)
    ctx.set_spaces(1, 2)
    for call in (lambda: ctx.dmrg_reference(8, 1), lambda: ctx.lcc_sweep(8, 1), lambda: ctx.energy()):
        with pytest.raises(mpslcc.MpsLccError) as e:
            call()
        assert e.value.status == 2 and str(e.value)
    assert len(ctx.mpo_bond_dims(mpslcc.MPO_H0)) == 5
    ctx.close()


def _header_structs(hdr):
    """Field names, in order, of every `typedef struct { ... } name;` in the header."""
    text = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for stmt in body.split(";"):
            stmt = stmt.strip()
            if not stmt:
                continue
            fp = re.search(r"\(\s*\*\s*(\w+)\s*\)", stmt)
            fields.append(fp.group(1) if fp else re.findall(r"\w+", stmt)[-1])
        out[name] = fields
    return out


@pytest.mark.parametrize("cname,pyname", [("mpslcc_opts", "Opts"), ("mpslcc_energies", "Energies"),
                                          ("mpslcc_stats", "Stats")])
def test_binding_structs_match_header_layout(mpslcc, cname, pyname, tmp_path):
    """The ctypes mirrors of the ABI structs have the header's fields, in order,
    at the offsets a C compiler gives them."""
    import shutil
    import subprocess
    hdr = open(os.path.join(ROOT, "include", "mpslcc.h")).read()
    fields = _header_structs(hdr)[cname]
    py = getattr(mpslcc, pyname)
    assert [f[0] for f in py._fields_] == fields
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpslcc.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({cname}));']
    lines += [f'  printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(py)
    assert got[1:] == [getattr(py, f).offset for f in fields]


def test_non_finite_integrals_are_rejected(mpslcc):
    """A NaN or infinity in h or V is an argument error; the context keeps
    working afterwards."""
    h, V = _integrals(3, 4)
    ctx = mpslcc.Context(device=-1)
    for bad in ("h", "V"):
        hb, Vb = h.copy(), V.copy()
        if bad == "h":
            hb[1, 1] = np.nan
        else:
            Vb[0, 0, 0, 0] = np.inf
        with pytest.raises(mpslcc.MpsLccError) as e:
            ctx.build_mpo(hb, Vb, n_elec=2, two_sz=0)
        assert e.value.status == 1 and "non-finite" in str(e.value)
    ctx.build_mpo(h, V, n_elec=2, two_sz=0)
    assert len(ctx.mpo_bond_dims(mpslcc.MPO_H)) == 4
    ctx.close()
