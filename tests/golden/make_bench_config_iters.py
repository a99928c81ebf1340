"""Writes bench_config_iters.json: the CPU oracle's converged PCG iteration counts for the
benchmark's own configuration, so that the GPU tests can compare iteration counts at full
size without re-running the slow FP64 oracle solves there.

Configuration (the inputs of bench.py, seed 1): 128 x 192 x 384 cells; conduction with
beta_Tcut, BE (Eqs. 2-4) by PCG (Fig. 1) to ||r|| <= 1e-10 ||W u^n|| at dt / dt_exp = 100,
1000 and 10000 with point Jacobi (PC1) and 8 x 8 x 8 block ILU0 (PC2, App. A); viscosity
at dt / dt_exp = 500 on each of the three Cartesian velocity components, both
preconditioners.  Only the oracle and the seeded input generators are called.

    python tests/golden/make_bench_config_iters.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1610_01265_gb300 import synth  # noqa: E402

DIMS = (128, 192, 384)
SEED = 1
RATIOS = (100.0, 1000.0, 10000.0)
VISC_RATIO = 500.0
RTOL = 1e-10
BLOCK = (8, 8, 8)


def main():
    nr, nth, nph = DIMS
    out = {"dims": list(DIMS), "seed": SEED, "rtol": RTOL, "block": list(BLOCK), "beta_tcut": True,
           "conduction": {}, "viscosity": {}}
    c = synth.conduction_case(nr, nth, nph, SEED)
    g = O.Grid(c["rf"], nth, nph)
    S, W = O.assemble_conduction(g, c["T"], c["bhat"], c["n"], beta_tcut=True)
    dte, _ = O.gershgorin_dt(g, S, W)
    out["conduction"]["dt_exp"] = dte
    for pc, name in ((O.PC_JACOBI, "jacobi"), (O.PC_BILU0, "bilu0")):
        for ratio in RATIOS:
            t0 = time.time()
            _, it, rel, st = O.be_pcg(g, S, W, c["T"], ratio * dte, pc=pc, block=BLOCK, rtol=RTOL, maxit=20000)
            out["conduction"][f"{name}_{int(ratio)}"] = {"iters": it, "relres": rel, "status": st}
            print(f"conduction {name} {ratio}: {it} iterations, relres {rel:.3e} ({time.time() - t0:.0f} s)",
                  flush=True)
    del S, W, c
    v = synth.viscosity_case(nr, nth, nph, SEED)
    g = O.Grid(v["rf"], nth, nph)
    S, W = O.assemble_viscosity(g, v["rho"], v["nu"])
    dtv, _ = O.gershgorin_dt(g, S, W)
    out["viscosity"]["dt_exp"] = dtv
    for pc, name in ((O.PC_JACOBI, "jacobi"), (O.PC_BILU0, "bilu0")):
        its = []
        for q in range(3):
            t0 = time.time()
            _, it, rel, st = O.be_pcg(g, S, W, v["v"][q], VISC_RATIO * dtv, pc=pc, block=BLOCK, rtol=RTOL,
                                      maxit=20000, pattern=7)
            its.append(it)
            print(f"viscosity {name} component {q}: {it} iterations, relres {rel:.3e} ({time.time() - t0:.0f} s)",
                  flush=True)
        out["viscosity"][f"{name}_{int(VISC_RATIO)}"] = {"iters": its}
    with open(os.path.join(HERE, "bench_config_iters.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
