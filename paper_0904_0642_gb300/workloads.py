"""Named synthetic workloads, run for a given number of sweeps (for
profilers and quick timing):

    python -m paper_0904_0642_gb300.workloads single --dims 32 32 32 32 --sweeps 10
    python -m paper_0904_0642_gb300.workloads ensemble --chains 256 --dims 8 8 8 8 --sweeps 2

single:   one hot-start lattice (FP32 12-real unless --storage), beta 6,
          2 hits, re-unitarised every 10 sweeps;
ensemble: --chains independent hot-start PBC chains of one shape in one
          fused launch per tick, beta_c ~ U[5.5, 6.5] from numpy seed 2009,
          seed_c = 5000 + c, re-unitarised every 10 sweeps.
--warm sweeps run first; --variant/--threads/--ctas fix the launch shape
(default: the autotuner's choice).  Prints the plaquette at the end.
"""
from __future__ import annotations

import argparse

import numpy as np

import paper_0904_0642_gb300 as su3

STORAGES = {"fp64_18": su3.SU3_FP64_18, "fp32_12": su3.SU3_FP32_12, "fp32_18": su3.SU3_FP32_18}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("kind", choices=["single", "ensemble"])
    ap.add_argument("--dims", type=int, nargs="+", default=[32, 32, 32, 32])
    ap.add_argument("--chains", type=int, default=256)
    ap.add_argument("--storage", choices=sorted(STORAGES), default="fp32_12")
    ap.add_argument("--sweeps", type=int, default=10)
    ap.add_argument("--warm", type=int, default=10)
    ap.add_argument("--variant", type=int, default=None)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--ctas", type=int, default=2)
    a = ap.parse_args(argv)
    storage = STORAGES[a.storage]
    if a.kind == "single":
        h = su3.Lattice(a.dims, beta=6.0, seed=20090406, hits=2, storage=storage, start=su3.SU3_START_HOT,
                        reunit_every=10)
    else:
        betas = np.random.default_rng(2009).uniform(5.5, 6.5, a.chains)
        cfgs = [su3.make_config(a.dims, beta=float(b), seed=5000 + c, storage=storage, start=su3.SU3_START_HOT,
                                hits=2, reunit_every=10) for c, b in enumerate(betas)]
        h = su3.Ensemble(cfgs)
    if a.variant is None:
        h.autotune()
    else:
        h.set_launch(a.threads, a.ctas, variant=a.variant)
    h.sweep(a.warm)
    h.sweep(a.sweeps)
    plaq = h.plaquette()[0] if a.kind == "single" else float(h.measure()[:, 0].mean())
    print(f"{a.kind} {'x'.join(map(str, a.dims))}: plaquette {plaq:.12f}")
    h.close()


if __name__ == "__main__":
    main()
