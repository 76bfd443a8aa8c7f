"""Writes the stored oracle values used by the GPU tests.

Calls only ``oracle/`` and ``synth/``.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import lcc  # noqa: E402


def main():
    out = {}
    c = synth.config(0)
    r = lcc.lcc_energies(c["h"], c["V"], c["n_alpha"], c["n_beta"], c["n_core"], c["n_active"])
    out["hubbard1d_L8_U4"] = dict(
        source="oracle.lcc.lcc_energies on synth.config(0): CAS-CI reference (Fink partition, "
               "Theory section), first order of Eq. 1 in projector form, E3 from Eq. 2 (n=1)",
        n_core=c["n_core"], n_active=c["n_active"],
        E0=r["E0"], E2=r["E2"], E3=r["E3"], Efci=r["Efci"], hylleraas=r["J"])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_energies.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
