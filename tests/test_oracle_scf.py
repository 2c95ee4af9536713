"""The oracle's one- and two-electron integrals and its RHF against a
textbook case: minimal-basis H2 (STO-3G, zeta = 1.24) at R = 1.4 bohr, whose
integral matrices, SCF energies and orbital energies are printed to four
decimals in Szabo & Ostlund (tests/golden/h2_sto3g.json).  Dropping a term of
any integral, a factor of the Fock matrix (F = h + J - K/2), or the energy
expression E = 1/2 tr(D(h + F)) + E_nuc moves one of these by far more than
the printed precision."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import scf

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "h2_sto3g.json")))
TOL = GOLD["printed_precision"]


def h2_basis():
    g = GOLD["sto3g_zeta_1p24"]
    a, d = list(g["exponents"]), list(g["coefficients"])
    return {"center": np.array(GOLD["geometry_bohr"], dtype=np.float64), "l": np.array([0, 0]),
            "nprim": np.array([3, 3]), "prim_off": np.array([0, 3]), "exps": np.array(a + a),
            "coefs": np.array(d + d), "atom": np.array([0, 1])}


def test_h2_sto3g_one_electron_integrals():
    b = h2_basis()
    Z = np.array([1.0, 1.0])
    S, T = oracle.overlap(b), oracle.kinetic(b)
    V = oracle.nuclear(b, Z, b["center"])
    V1 = oracle.nuclear(b, np.array([1.0, 0.0]), b["center"])  # attraction to nucleus 1 only
    g = GOLD["one_electron"]
    got = {"S12": S[0, 1], "T11": T[0, 0], "T12": T[0, 1], "V1_11": V1[0, 0], "V1_12": V1[0, 1],
           "V1_22": V1[1, 1], "Hcore11": T[0, 0] + V[0, 0], "Hcore12": T[0, 1] + V[0, 1]}
    for k, v in got.items():
        assert abs(v - g[k]) <= TOL, (k, v, g[k])
    assert abs(S[0, 0] - 1.0) < 1e-12 and abs(S[1, 1] - 1.0) < 1e-12


def test_h2_sto3g_two_electron_integrals():
    b = h2_basis()

    def eri(i, j, k, l):
        return float(np.asarray(oracle.shell_eri(b, i, j, k, l)).ravel()[0])

    g = GOLD["two_electron"]
    got = {"11_11": eri(0, 0, 0, 0), "11_22": eri(0, 0, 1, 1), "21_11": eri(1, 0, 0, 0),
           "21_21": eri(1, 0, 1, 0)}
    for k, v in got.items():
        assert abs(v - g[k]) <= TOL, (k, v, g[k])


@pytest.mark.parametrize("guess", ["core", "zero"])
def test_h2_sto3g_rhf(guess):
    b = h2_basis()
    Z = np.array([1.0, 1.0])
    D0 = None if guess == "core" else np.zeros((2, 2))
    r = scf.rhf(b, Z, b["center"], nocc=1, tau=0.0, D0=D0)
    g = GOLD["scf"]
    assert abs(r["electronic"] - g["electronic_energy"]) <= TOL
    assert abs(r["energy"] - g["total_energy"]) <= TOL
    assert np.allclose(r["eps"], g["orbital_energies"], atol=TOL)
    assert abs(scf.nuclear_repulsion(Z, b["center"]) - 1.0 / 1.4) < 1e-15
    # closed shell: tr(D S) = number of electrons
    assert abs(np.sum(r["D"] * oracle.overlap(b)) - 2.0) < 1e-10
