"""The learned-guess experiment: RHF on seeded conformations (C8-C16 alkanes,
(H2O)8-16 clusters; 6-31G(d)-shaped synthetic basis; FP64 J/K; DIIS;
convergence 1e-8 Eh) from the SAD guess; the atom-pair MLP is trained on the
converged densities of the training conformations with the library's
forward/backward kernels; on the held-out conformations the SCF is rerun
from the MLP guess and compared with SAD by iterations, time and energy.

    python -m paper_2407_21445_gb300.train_guess --n 500 --train 400 --out DIR

Writes DIR/report.json and DIR/mlp_params.npz (network, feature normaliser).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

import molgen

from . import guess as G
from .scf import RHF, sad_guess


def split(n: int = 500, ntrain: int = 400, seed: int = 0):
    """The seeded train / held-out split of the n conformations."""
    rng = np.random.Generator(np.random.PCG64(50_000 + seed))
    order = rng.permutation(n)
    return sorted(order[:ntrain].tolist()), sorted(order[ntrain:].tolist())


def run(n: int, ntrain: int, out: str, epochs: int, seed: int = 0, tau: float = 1e-10, log=print):
    os.makedirs(out, exist_ok=True)
    table = molgen.basis_set("dz", seed)
    mols = molgen.scf_conformations(n, seed)
    train_idx, test_idx = split(n, ntrain, seed)
    rec = {}
    feats, targs, masks = [], [], []
    t0 = time.time()
    for i in range(n):
        mol = mols[i]
        basis = molgen.make_basis(mol, table)
        rhf = RHF(mol.Z.astype(float), mol.coords, basis, tau=tau)
        ts = time.time()
        Ds = sad_guess(mol, table)
        r = rhf.run(Ds)
        torch.cuda.synchronize()
        rec[i] = dict(natom=mol.natom, nbf=int(rhf.S.shape[0]), sad_E=r.energy, sad_it=r.iterations,
                      sad_conv=r.converged, sad_t=time.time() - ts)
        if i in set(train_idx):
            pairs, frames, f = G.pair_frames(mol)
            T, M = G.blocks_to_local(r.D.cpu().numpy() - Ds.cpu().numpy(), mol, basis, pairs, frames)
            feats.append(f)
            targs.append(T)
            masks.append(M)
        if i % 25 == 0:
            log(f"scf {i}/{n} nbf={rec[i]['nbf']} it={r.iterations} E={r.energy:.8f} ({time.time() - t0:.0f}s)")
    F, T, M = np.concatenate(feats), np.concatenate(targs), np.concatenate(masks)
    log(f"training samples {F.shape[0]}")
    lg = G.LearnedGuess(hidden=128, max_batch=8192, seed=seed)
    lg.fit_normaliser(F)
    tt = time.time()
    hist = lg.train(F, T, M, epochs=epochs, batch=4096, lr=2e-3, seed=seed, log=log)
    train_s = time.time() - tt
    res = []
    for i in test_idx:
        mol = mols[i]
        basis = molgen.make_basis(mol, table)
        rhf = RHF(mol.Z.astype(float), mol.coords, basis, tau=tau)
        ts = time.time()
        D0 = lg.guess(mol, basis, rhf, sad_guess(mol, table).cpu().numpy())
        r = rhf.run(D0)
        torch.cuda.synchronize()
        rr = dict(rec[i])
        rr.update(mlp_E=r.energy, mlp_it=r.iterations, mlp_conv=r.converged, mlp_t=time.time() - ts,
                  dE=abs(r.energy - rec[i]["sad_E"]))
        res.append(rr)
    sad_it = np.array([r["sad_it"] for r in res], float)
    mlp_it = np.array([r["mlp_it"] for r in res], float)
    report = {
        "conformations": n, "train": ntrain, "held_out": len(test_idx), "basis": "6-31G(d)-shaped synthetic",
        "convergence": "|dE| < 1e-8 Eh and max |X^T (FDS - SDF) X| < 1e-6",
        "held_out_mean_iterations": {"sad": float(sad_it.mean()), "mlp": float(mlp_it.mean())},
        "iteration_reduction": float(1.0 - mlp_it.mean() / sad_it.mean()),
        "held_out_mean_time_s": {"sad": float(np.mean([r["sad_t"] for r in res])),
                                 "mlp": float(np.mean([r["mlp_t"] for r in res]))},
        "max_abs_energy_diff_Eh": float(max(r["dE"] for r in res)),
        "all_converged": bool(all(r["sad_conv"] and r["mlp_conv"] for r in res)),
        "train_mean_sad_iterations": float(np.mean([rec[i]["sad_it"] for i in train_idx])),
        "training_loss_first_last": [float(hist[0]), float(hist[-1])], "training_seconds": train_s,
        "epochs": epochs, "samples": int(F.shape[0]), "per_molecule": res,
    }
    with open(os.path.join(out, "report.json"), "w") as f:
        json.dump(report, f, indent=1)
    np.savez(os.path.join(out, "mlp_params.npz"), params=lg.net.params(), mu=lg.mu, sd=lg.sd)
    return report


def sensitivity(params: str, out: str, n: int = 500, ntrain: int = 400, nmol: int = 10, seed: int = 0,
                tau: float = 1e-10, scales=(1.0, 0.3, 0.1, 0.03, 0.01, 1e-3, 1e-4), log=print):
    """How accurate must a guess be?  On the first nmol held-out conformations
    (same seeded split as run()): SCF from the idempotent projection of
    D_conv + s (D_SAD - D_conv) for each scale s, the Frobenius errors
    |D0 - D_conv| of the SAD and the trained-MLP guesses, and the MLP's
    iterations.  Writes out/sensitivity.json."""
    os.makedirs(out, exist_ok=True)
    table = molgen.basis_set("dz", seed)
    mols = molgen.scf_conformations(n, seed)
    test_idx = split(n, ntrain, seed)[1][:nmol]
    lg = G.LearnedGuess.load(params)
    rows = []
    for i in test_idx:
        mol = mols[i]
        basis = molgen.make_basis(mol, table)
        rhf = RHF(mol.Z.astype(float), mol.coords, basis, tau=tau)
        Ds = sad_guess(mol, table)
        r = rhf.run(Ds)
        Dc = r.D
        Dm = lg.guess(mol, basis, rhf, Ds.cpu().numpy())
        rm = rhf.run(Dm)
        Dsp = G.project_idempotent(Ds, rhf.S, rhf.X, rhf.nocc)
        row = dict(index=i, nbf=int(rhf.S.shape[0]), sad_it=r.iterations, mlp_it=rm.iterations,
                   err_sad=float(torch.linalg.norm(Ds - Dc)), err_sad_projected=float(torch.linalg.norm(Dsp - Dc)),
                   err_mlp=float(torch.linalg.norm(Dm - Dc)), scaled={})
        for sc in scales:
            D0 = G.project_idempotent(Dc + sc * (Ds - Dc), rhf.S, rhf.X, rhf.nocc)
            rs = rhf.run(D0)
            row["scaled"][str(sc)] = dict(it=rs.iterations, err=float(torch.linalg.norm(D0 - Dc)),
                                          dE=abs(rs.energy - r.energy))
        rows.append(row)
        log(f"{i}: sad {row['sad_it']} mlp {row['mlp_it']} err sad {row['err_sad']:.3g} mlp {row['err_mlp']:.3g} "
            + " ".join(f"{k}:{v['it']}" for k, v in row["scaled"].items()))
    summ = {"mean_sad_it": float(np.mean([r["sad_it"] for r in rows])),
            "mean_mlp_it": float(np.mean([r["mlp_it"] for r in rows])),
            "mean_err_sad": float(np.mean([r["err_sad"] for r in rows])),
            "mean_err_mlp": float(np.mean([r["err_mlp"] for r in rows])),
            "mean_it_by_scale": {str(sc): float(np.mean([r["scaled"][str(sc)]["it"] for r in rows])) for sc in scales},
            "mean_err_by_scale": {str(sc): float(np.mean([r["scaled"][str(sc)]["err"] for r in rows]))
                                  for sc in scales},
            "rows": rows}
    with open(os.path.join(out, "sensitivity.json"), "w") as f:
        json.dump(summ, f, indent=1)
    return summ


def evaluate(params_npz: str, out: str, n: int = 500, ntrain: int = 400, limit: int = 0, seed: int = 0,
             tau: float = 1e-10, log=print):
    """Held-out comparison with a trained network and no retraining: per
    held-out conformation the SCF from SAD and from the MLP guess, iterations
    and wall time (guess construction, featurisation, network, projection and
    SCF, the GPU synchronised) and the energy difference."""
    os.makedirs(out, exist_ok=True)
    table = molgen.basis_set("dz", seed)
    mols = molgen.scf_conformations(n, seed)
    _, test_idx = split(n, ntrain, seed)
    if limit > 0:
        test_idx = test_idx[:limit]
    lg = G.LearnedGuess.load(params_npz)
    sad_guess(mols[test_idx[0]], table)  # atomic densities cached outside the timings
    res = []
    for i in test_idx:
        mol = mols[i]
        basis = molgen.make_basis(mol, table)
        out_i = {"natom": mol.natom}
        for name in ("sad", "mlp"):
            rhf = RHF(mol.Z.astype(float), mol.coords, basis, tau=tau)
            torch.cuda.synchronize()
            ts = time.time()
            Ds = sad_guess(mol, table)
            D0 = Ds if name == "sad" else lg.guess(mol, basis, rhf, Ds.cpu().numpy())
            r = rhf.run(D0)
            torch.cuda.synchronize()
            out_i.update({f"{name}_t": time.time() - ts, f"{name}_it": r.iterations, f"{name}_E": r.energy,
                          f"{name}_conv": r.converged})
        out_i["dE"] = abs(out_i["mlp_E"] - out_i["sad_E"])
        res.append(out_i)
    rep = {"params": params_npz, "held_out": len(res),
           "mean_iterations": {k: float(np.mean([r[f"{k}_it"] for r in res])) for k in ("sad", "mlp")},
           "mean_wall_s": {k: float(np.mean([r[f"{k}_t"] for r in res])) for k in ("sad", "mlp")},
           "max_abs_energy_diff_Eh": float(max(r["dE"] for r in res)),
           "all_converged": bool(all(r["sad_conv"] and r["mlp_conv"] for r in res)), "per_molecule": res}
    rep["iteration_reduction"] = 1.0 - rep["mean_iterations"]["mlp"] / rep["mean_iterations"]["sad"]
    rep["wall_reduction"] = 1.0 - rep["mean_wall_s"]["mlp"] / rep["mean_wall_s"]["sad"]
    with open(os.path.join(out, "evaluate.json"), "w") as f:
        json.dump(rep, f, indent=1)
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--evaluate", default=None, metavar="PARAMS_NPZ",
                    help="instead of training: held-out SCF iterations and wall time with a trained network")
    ap.add_argument("--limit", type=int, default=0, help="--evaluate: first LIMIT held-out conformations (0 = all)")
    ap.add_argument("--sensitivity", default=None, metavar="PARAMS_NPZ",
                    help="instead of training: guess-accuracy study with a trained network")
    ap.add_argument("--n", type=int, default=500)
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="guess_run")
    a = ap.parse_args()
    if a.evaluate:
        rep = evaluate(a.evaluate, a.out, a.n, a.train, a.limit, seed=a.seed)
        print(json.dumps({k: v for k, v in rep.items() if k != "per_molecule"}))
        return
    if a.sensitivity:
        rep = sensitivity(a.sensitivity, a.out, a.n, a.train, seed=a.seed)
        print(json.dumps({k: v for k, v in rep.items() if k != "rows"}))
        return
    rep = run(a.n, a.train, a.out, a.epochs, a.seed)
    print(json.dumps({k: v for k, v in rep.items() if k != "per_molecule"}))


if __name__ == "__main__":
    main()
