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

omega_200atom_rsh.json: the timed 200-atom case (seed 2, 100 heavy + 100 H,
nao 1900, nocc 380; K operator (0.222 + 0.778 erf(0.2 r))/r, c_x = 1, 40 eV
window): the 15 lowest excitation energies from the oracle's matrix-free block
Davidson (Sec. 3.3) with a block of 30 and residual 1e-7, and the oracle's A X
for the two seeded unit trial vectors synth.random_trial_block(2024, 2, ...)
on sampled entries: one whole occupied row i per vector and 128 seeded (i, a)
positions.  Also the wall time of the run and the threads it used (the
machine that wrote the file is named in it).

Run: python tests/golden/make_golden.py [tda|tddft|props|cfg2]   (default: tda)
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


# the timed 200-atom case: range-separated exchange, 15 states, block 30
CFG2 = dict(cx=1.0, ka=0.222, kb=0.778, omega=0.2)
CFG2_X_SEED = 2024
CFG2_ROWS = (7, 301)          # whole occupied rows i of AX, one per vector
CFG2_SAMPLES = 128            # seeded (i, a) positions per vector


def cfg2_sample_positions(nocc, nvir):
    """The seeded (i, a) positions stored per vector (shared with the GPU test)."""
    rng = np.random.default_rng(CFG2_X_SEED + 1)
    return rng.integers(0, nocc, size=CFG2_SAMPLES), rng.integers(0, nvir, size=CFG2_SAMPLES)


def main_cfg2():
    import platform
    import time
    t_all = time.perf_counter()
    mol = synth.molecule_200()
    t0 = time.perf_counter()
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, CFG2["cx"],
                  CFG2["ka"], CFG2["kb"], CFG2["omega"], window_ev=40.0)
    t_build = time.perf_counter() - t0
    print("build %.1f s" % t_build, flush=True)
    X = synth.random_trial_block(CFG2_X_SEED, 2, mol.nocc, mol.nvir)
    t0 = time.perf_counter()
    AX = tda.matvec(f, X)
    t_mv = time.perf_counter() - t0
    ii, aa = cfg2_sample_positions(mol.nocc, mol.nvir)
    t0 = time.perf_counter()
    res = tda.solve(f, 15, block=30, tol=1e-7)
    t_solve = time.perf_counter() - t0
    print("solve %.1f s, %d iterations, %d matvecs" % (t_solve, res.niter, res.nmatvec), flush=True)
    out = {"source": "oracle matrix-free block Davidson (Sec. 3.3) of the TDA-risp matrix (Sec. 2, Eq. "
                     "TDA-risp) with range-separated exchange (Sec. 3.2, Eqs. RSH and K_mia_RSH), and the "
                     "oracle's matrix-free A X",
           "molecule": "synth.molecule_200(): seed 2, 100 heavy + 100 H, nao 1900, nocc 380",
           "options": CFG2, "window_ev": 40.0, "nstates": 15, "block": 30, "tol": 1e-7,
           "omega": [float(x) for x in res.omega], "resid": [float(x) for x in res.resid],
           "converged": bool(res.converged), "niter": int(res.niter), "nmatvec": int(res.nmatvec),
           "nrestart": int(res.nrestart),
           "ax": {"x_seed": CFG2_X_SEED, "m": 2,
                  "generator": "synth.random_trial_block(x_seed, m, nocc, nvir)",
                  "rows": [{"vector": k, "i": CFG2_ROWS[k], "values": [float(v) for v in AX[k, CFG2_ROWS[k]]]}
                           for k in range(2)],
                  "samples": {"i": [int(i) for i in ii], "a": [int(a) for a in aa],
                              "values": [[float(AX[k, i, a]) for i, a in zip(ii, aa)] for k in range(2)]},
                  "max_abs": [float(np.abs(AX[k]).max()) for k in range(2)]},
           "timing": {"build_s": t_build, "matvec_2_vectors_s": t_mv, "solve_s": t_solve,
                      "total_s": time.perf_counter() - t_all, "threads": os.cpu_count(),
                      "machine": "%s, %s" % (platform.machine(), platform.processor() or "cpu")}}
    with open(os.path.join(HERE, "omega_200atom_rsh.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(res.omega)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "tda"
    {"tda": main, "tddft": main_tddft, "props": main_props, "cfg2": main_cfg2}[which]()
