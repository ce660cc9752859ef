"""Writes prec_n2048_m256_oracle_misfit.txt: the FP64 oracle's misfit Phi after
each of the first epochs of the precision workload (n = 2048, m = 256,
N = 4096, B = 256, L = 3 bilinear, Poisson peak 1e5; Sec. 3 sweep from the
flat object and the blurred, dp_avg-scaled probe of Sec. 4.1).

The tensor-core and FP32 variants of the library are timed until their own
end-of-epoch misfit reaches the oracle's last value (time-to-oracle-misfit).
Only the oracle and the seeded input generators run here.  About 15 minutes
single-threaded:  python tests/golden/make_prec_target.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

NAME = "prec_n2048_m256"


def main():
    w = synth.make_workload(NAME)
    p = w.params
    E = p["epochs"]
    d = O.forward_intensity(w.q_true, w.z_true, w.pos)
    rng = np.random.Generator(np.random.PCG64(p["noise_seed"]))
    d = synth.poisson_noise(d, p["peak"], rng).astype(np.float32).astype(np.float64)
    a = np.sqrt(np.maximum(d, 0.0))
    z = np.ones((p["n"], p["n"]), dtype=np.complex128)
    q = O.dp_avg_scale(w.q_init_blurred, d)
    orders = synth.epoch_orders(len(w.pos), E, p["order_seed"])
    prm = O.Params(alpha=p["alpha"], levels=p["levels"], minibatch=p["minibatch"], prolong=p["prolong"])
    phis = []
    t0 = time.time()
    for e in range(E):
        z, q = O.run_epochs(z, q, w.pos, a, [orders[e]], prm, eval_misfit=False)[:2]
        phis.append(O.misfit(q, z, w.pos, a))
        print(f"epoch {e + 1}: Phi = {phis[-1]:.10e}  ({time.time() - t0:.0f} s)", flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{NAME}_oracle_misfit.txt")
    with open(out, "w") as f:
        f.write(f"# FP64 oracle misfit Phi = 1/2 sum_k ||Q P_k z - R_k||^2 (Sec. 2.1) after each epoch of the\n")
        f.write(f"# {NAME} workload: n={p['n']} m={p['m']} N={len(w.pos)} B={p['minibatch']} L={p['levels']} "
                f"{p['prolong']}, alpha={p['alpha']}, peak={p['peak']:g}, seed={p['seed']}; orders from\n")
        f.write("# synth.epoch_orders, intensities from oracle.forward_intensity + synth.poisson_noise\n")
        f.write("# (rounded to float32).  Written by tests/golden/make_prec_target.py.\n")
        f.write("# epoch phi\n")
        for e, v in enumerate(phis):
            f.write(f"{e + 1} {v:.12e}\n")


if __name__ == "__main__":
    main()
