"""Write the stored expected values under tests/golden/ from the CPU oracle only.

omega_24atom.json: the 5 lowest TDA-risp excitation energies (Hartree) of the
24-atom seeded molecule (10 heavy + 14 H, nao 210, nocc 42) by dense eigh of the
explicit matrix A_{ia,jb} = (e_a - e_i) d d + 2 (ia|jb) - c_x (ij|ab)  (paper Sec. 2,
Eq. TDA-risp; RI through the minimal aux basis, Sec. 2 Eq. RI and Sec. 3.2), for a
global hybrid (c_x = 0.25, 40 eV window) and a range-separated case
((0.222 + 0.778 erf(0.2 r))/r, c_x = 1).

omega_tddft_24atom.json: the 5 lowest full TDDFT-risp excitation energies of the
same molecule and cases (Sec. 2, Eqs. tddft and hessian, with A + B = D + 4 (ia|jb)
- c_x [(ib|ja) + (ij|ab)] and A - B = D + c_x [(ib|ja) - (ij|ab)]) by the dense
symmetric-form solve of the oracle.

oscillator_24atom.json: the oscillator strengths f = 2/3 Omega |mu|^2 (Sec. 2,
Eqs. oscillator_strength and transition) of those states, TDA (unit-norm X) and
full TDDFT (X+Y with (X+Y).(X-Y) = 1), dipoles about the coordinate origin.

Run: python tests/golden/make_golden.py [tda|tddft|props]   (default: tda)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np
import scipy.linalg

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tda  # noqa: E402
from paper_2603_29257_gb300 import synth  # noqa: E402

CASES = {
    "hybrid": dict(cx=0.25, ka=1.0, kb=0.0, omega=0.0),
    "rsh": dict(cx=1.0, ka=0.222, kb=0.778, omega=0.2),
}


def main():
    mol = synth.molecule_24()
    out = {"source": "oracle dense eigh of the explicit TDA-risp matrix (Sec. 2, Eq. TDA-risp)",
           "molecule": "synth.molecule_24(): seed 1, 10 heavy + 14 H, nao 210, nocc 42",
           "window_ev": 40.0, "nstates": 5, "cases": {}}
    for name, op in CASES.items():
        f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, op["cx"],
                      op["ka"], op["kb"], op["omega"], window_ev=40.0)
        A = tda.explicit_A(f)
        w = scipy.linalg.eigh(A, eigvals_only=True, subset_by_index=[0, 4], driver="evr")
        out["cases"][name] = {"options": op, "omega": [float(x) for x in w]}
        print(name, w)
    with open(os.path.join(HERE, "omega_24atom.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def main_tddft():
    mol = synth.molecule_24()
    out = {"source": "oracle dense symmetric-form solve of full TDDFT-risp (Sec. 2, Eqs. tddft and hessian)",
           "molecule": "synth.molecule_24(): seed 1, 10 heavy + 14 H, nao 210, nocc 42",
           "window_ev": 40.0, "nstates": 5, "cases": {}}
    for name, op in CASES.items():
        f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, op["cx"],
                      op["ka"], op["kb"], op["omega"], window_ev=40.0, tddft=True)
        w, _, _ = tda.tddft_dense(f, 5)
        out["cases"][name] = {"options": op, "omega": [float(x) for x in w]}
        print(name, w)
    with open(os.path.join(HERE, "omega_tddft_24atom.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def main_props():
    mol = synth.molecule_24()
    out = {"source": "oracle: dense TDA eigh and dense full TDDFT solve, then the oracle's transition dipoles "
                     "(Sec. 2, Eqs. oscillator_strength, transition)",
           "molecule": "synth.molecule_24(): seed 1, 10 heavy + 14 H, nao 210, nocc 42",
           "window_ev": 40.0, "nstates": 5, "cases": {}}
    for name, op in CASES.items():
        f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, op["cx"],
                      op["ka"], op["kb"], op["omega"], window_ev=40.0, tddft=True)
        w, V = scipy.linalg.eigh(tda.explicit_A(f), subset_by_index=[0, 4], driver="evr")
        X = tda.fix_sign(V.T).reshape(5, f.nocc, f.nvir)
        f_tda = tda.oscillator_strengths(w, tda.transition_dipoles(mol.xyz, mol.shells, mol.C, mol.nocc, X))
        wd, XpY, _ = tda.tddft_dense(f, 5)
        f_rpa = tda.oscillator_strengths(wd, tda.transition_dipoles(mol.xyz, mol.shells, mol.C, mol.nocc, XpY))
        out["cases"][name] = {"options": op, "omega_tda": [float(x) for x in w], "f_tda": [float(x) for x in f_tda],
                              "omega_tddft": [float(x) for x in wd], "f_tddft": [float(x) for x in f_rpa]}
        print(name, f_tda, f_rpa)
    with open(os.path.join(HERE, "oscillator_24atom.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "tda"
    {"tda": main, "tddft": main_tddft, "props": main_props}[which]()
