"""Complex-Langevin runs with the exact fermion drift (Sec. 4.1 set-up).

    python -m paper_1707_08874_gb300.run_langevin --Ns 8 --Nt 4 --beta 5.0 --steps 200 \
        [--precision fp64_emu|fp64|mixed|fp32] [--batch B] [--n-cool 5] [--out run.jsonl]
        [--lt 30 --therm 5] [--reunit] [--hist 40]

Each line of output is one step of replica 0 (and the replica means): Langevin
time, step size, K_max, plaquettes, Polyakov loops, condensate, unitarity
norm.  The adaptive step follows eps = min(eps_max, kappa / K_max); with
--kappa 0 (default) kappa is set after --calib steps at eps_max to
eps_max * mean(K_max) of those steps.  With --lt the run goes on until the
Langevin time of replica 0 reaches lt (Sec. 4.1: 30 Lt, of which 5 are
thermalisation, --therm).  The last line is a summary of the measurements
after thermalisation, over all replicas: means with errors from binning the
steps of every chain into 10 blocks, and with --hist N the histograms of the
chiral condensate and the Polyakov loop (real and imaginary parts, N bins;
Sec. 4.1 judges the validity of a run by exponentially decaying tails) with the
fraction of samples beyond 3 and 4 standard deviations beside the Gaussian
fractions 2.7e-3 and 6.3e-5.
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--Ns", type=int, default=8)
    ap.add_argument("--Nt", type=int, default=4)
    ap.add_argument("--beta", type=float, default=5.0)
    ap.add_argument("--m", type=float, default=0.05)
    ap.add_argument("--mu", type=float, default=0.25)
    ap.add_argument("--nf", type=float, default=1.0)
    ap.add_argument("--eps-max", type=float, default=1e-3)
    ap.add_argument("--kappa", type=float, default=0.0)
    ap.add_argument("--calib", type=int, default=10)
    ap.add_argument("--n-cool", type=int, default=5)
    ap.add_argument("--alpha-cool", type=float, default=0.05)
    ap.add_argument("--renorm-det", action="store_true", help="U <- U / det(U)^(1/3) after each update")
    ap.add_argument("--reunit", action="store_true", help="project the links onto SU(3) after each update")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lt", type=float, default=0.0, help="run until Langevin time lt (overrides --steps)")
    ap.add_argument("--therm", type=float, default=0.0, help="Langevin time discarded before the summary")
    ap.add_argument("--hist", type=int, default=0, help="bins of the condensate / Polyakov-loop histograms")
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--seed", type=int, default=1707)
    ap.add_argument("--precision", choices=["fp64", "fp64_emu", "mixed", "fp32"], default="fp64_emu")
    ap.add_argument("--start", choices=["random", "su3", "cold"], default="random")
    ap.add_argument("--out", default=None)
    ap.add_argument("--checkpoint", default=None, help="write a checkpoint here at the end (and every --every steps)")
    ap.add_argument("--every", type=int, default=0)
    ap.add_argument("--resume", default=None, help="continue from this checkpoint")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from . import binding as B
    from . import checkpoint
    from . import inputs

    prec = {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_BF16X3,
            "fp32": B.CL_MIXED_FP32}[args.precision]
    plan = B.Plan.analyze(args.Ns, args.Nt, args.batch, prec)
    if args.start == "cold":
        U0 = np.stack([inputs.unit_links(args.Ns, args.Nt)] * args.batch)
    else:
        U0 = inputs.random_links(args.Ns, args.Nt, seed=args.seed, batch=args.batch,
                                 sigma_im=0.1 if args.start == "random" else 0.0)
    state0 = np.zeros((args.batch, 4))
    if args.resume:
        U0, state0, saved = checkpoint.load(args.resume)
        args.kappa = saved.get("kappa", args.kappa)
    U = torch.from_numpy(U0).to("cuda")
    state = torch.from_numpy(state0).to("cuda")
    obs = torch.zeros((args.batch, B.OBS_LEN), dtype=torch.float64, device="cuda")
    prm = dict(beta=args.beta, m=args.m, mu=args.mu, nf=args.nf, eps_max=args.eps_max, kappa=args.kappa,
               alpha_cool=args.alpha_cool, seed=args.seed, n_cool=args.n_cool, fermions=1,
               renorm_det=int(args.renorm_det), reunit=int(args.reunit))
    out = open(args.out, "w") if args.out else sys.stdout
    kcal = []
    keys = ("plaq_s", "plaq_t", "poly", "poly_inv", "condensate", "density")
    hist = []  # per step after thermalisation: [replica][observable] complex
    t0 = time.time()
    step = 0
    while (step < args.steps) if args.lt <= 0 else (float(state[0, 0].item()) < args.lt):
        plan.langevin_step(U, prm, state, obs)
        o = obs.cpu().numpy()
        st, _ = plan.get_status()
        rows = [B.obs_dict(r) for r in o]
        if prm["kappa"] <= 0 and step < args.calib:
            kcal.append(float(np.mean([r["kmax"] for r in rows])))
            if step == args.calib - 1:
                prm["kappa"] = args.eps_max * float(np.mean(kcal))
        rec = {"step": step + 1, "status": st, "wall_s": round(time.time() - t0, 3)}
        r0 = rows[0]
        for k in ("t", "eps", "kmax", "unitarity"):
            rec[k] = r0[k]
        for k in ("plaq_s", "plaq_t", "poly", "poly_inv", "condensate", "density"):
            rec[k] = [r0[k].real, r0[k].imag]
            if args.batch > 1:
                m = np.mean([r[k] for r in rows])
                rec[k + "_mean"] = [m.real, m.imag]
        print(json.dumps(rec), file=out, flush=True)
        if r0["t"] >= args.therm:
            hist.append([[r[k] for k in keys] for r in rows])
        step += 1
        if st != B.CL_OK:
            print(json.dumps({"error": B.error_string(st), "step": step}), file=out, flush=True)
            break
        if args.checkpoint and args.every and step % args.every == 0:
            checkpoint.save(args.checkpoint, U, state, prm)
    if args.checkpoint:
        checkpoint.save(args.checkpoint, U, state, prm)
    if hist:
        print(json.dumps(summary(np.array(hist), keys, args.hist)), file=out, flush=True)
    plan.close()


def summary(h, keys, bins):
    """Means after thermalisation over all chains with binned errors (each
    chain's steps in 10 consecutive blocks), and histograms of the condensate
    and the Polyakov loop.  h: [steps, replicas, observables] complex."""
    import numpy as np
    nsteps, nrep, _ = h.shape
    nb = 10 if nsteps >= 10 else 1
    L = nsteps // nb * nb
    rec = {"summary": True, "steps": int(nsteps), "replicas": int(nrep)}
    for j, k in enumerate(keys):
        x = h[:L, :, j]
        blocks = x.reshape(nb, L // nb, nrep).mean(1).reshape(-1)  # block means of every chain
        m = blocks.mean()
        rec[k] = {"mean": [float(m.real), float(m.imag)],
                  "err": [float(np.std(blocks.real, ddof=1) / np.sqrt(len(blocks))) if len(blocks) > 1 else None,
                          float(np.std(blocks.imag, ddof=1) / np.sqrt(len(blocks))) if len(blocks) > 1 else None]}
    if bins > 0:
        for k in ("condensate", "poly"):
            x = h[:, :, keys.index(k)].reshape(-1)
            for part, v in (("re", x.real), ("im", x.imag)):
                cnt, edges = np.histogram(v, bins=bins)
                sd = v.std()
                z = np.abs(v - v.mean()) / sd if sd > 0 else np.zeros_like(v)
                rec["hist_%s_%s" % (k, part)] = {"counts": cnt.tolist(), "edges": [float(e) for e in edges],
                                                "frac_beyond_3sd": float((z > 3).mean()),
                                                "frac_beyond_4sd": float((z > 4).mean())}
    return rec


if __name__ == "__main__":
    main()
