"""Write the reference shower statistics of the oracle's untabulated transport.

    python tests/golden/make_exact_showers.py [threads]

Runs only the FP64 oracle (oracle/), in its untabulated mode: cross sections
from their formulas at each track's energy, range and continuous loss by
quadrature and root finding, every final state by rejection from its DCS.
Writes, per workload, the number of showers and the mean and variance of the
per-event deposit of every layer and every material, for the tests that
compare the tabulated transport (oracle and GPU) with it.  The seed differs
from the workloads' default one, so the stored sample is independent of the
samples the tests draw.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import shower_stats  # noqa: E402
from paper_2005_00949_gb300 import workloads as W  # noqa: E402

SEED = W.DEFAULT_SEED ^ 0x5A5A5A5A

# (file, workload, description)
CASES = [
    ("exact_showers_e-1GeV_PbPS50.txt", lambda: W.pbps_electrons(200_000, 1000.0),
     "200000 x 1 GeV e- on 50 x (2 mm Pb + 5 mm polystyrene), 40x40 cm, cuts 1 MeV"),
    ("exact_showers_e-10GeV_PbPS50.txt", lambda: W.pbps_electrons(65_536, 10_000.0),
     "65536 x 10 GeV e- on 50 x (2 mm Pb + 5 mm polystyrene), 40x40 cm, cuts 1 MeV"),
    ("exact_showers_e-100GeV_WSi50.txt", lambda: W.wsi_cells(2048, 100_000.0),
     "2048 x 100 GeV e- on 50 x (3 mm W + 0.5 mm Si), 40x40 cm, entry points uniform over the "
     "central 4x4 cells of 1.25 cm, cuts 0.5 MeV"),
    ("exact_showers_e-10GeV_PbLAr50_4T_msc.txt",
     lambda: W.with_msc(W.with_field(W.pblar_testem3(8192, 10_000.0), 4.0, 1)),
     "8192 x 10 GeV e- on 50 x (2.3 mm Pb + 5.7 mm liquid argon), 40x40 cm, 4 T along y, "
     "multiple scattering, cuts 0.1 MeV (gamma) / 1 MeV (e)"),
]


def main():
    nthr = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    only = sys.argv[2:] or None
    for name, make, desc in CASES:
        if only and name not in only:
            continue
        wl = make()
        wl.seed = SEED
        t = time.time()
        r = oracle.Oracle(wl, exact=True).transport(n_threads=nthr)
        dt = time.time() - t
        s = shower_stats.summarize(r["edep"], wl.n_layers)
        steps = int(r["counts"][:, 0].sum())
        shower_stats.write(os.path.join(HERE, name), s, [
            "Untabulated FP64 oracle (Oracle(wl, exact=True)): reference shower statistics.",
            f"Workload: {desc}.",
            f"Seed {SEED:#x}; {steps} track steps; {nthr} threads, {dt:.0f} s.",
            "Written by tests/golden/make_exact_showers.py, which runs only oracle/.",
            "Per layer (absorber + gap) and per material (summed over layers):",
            "mean and variance (ddof=1) of the per-event deposit, MeV.",
        ])
        print(name, steps, f"{dt:.1f} s", flush=True)


if __name__ == "__main__":
    main()
