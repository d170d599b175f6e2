"""Write the stored expected values that the GPU tests and the benchmark read.

Calls only the FP64 oracle (oracle/) on seeded synthetic inputs (synth/):
  small_oracle_cost.json  cost history of the 64x64x16 one-coil workload, 50 NCG-MLS-IC(0)
                          iterations (N_ls = 5): the target of the time-to-cost figure.
  full8_oracle_cost.json  cost history of the 64x64x32 eight-coil volume drawn by the full
                          workload's recipe, 100 NCG-MLS-IC(0) iterations (N_ls = 5): the
                          eight-coil time-to-cost target (about 90 s on 8 host threads).
Run:  python tests/golden/make_golden.py [small|full8]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle, set_threads  # noqa: E402
from synth import full8_small_config, small_config  # noqa: E402

SOURCE = "FP64 oracle (oracle/fm_oracle.c), NCG-MLS-IC(0), N_ls = 5, from the Eq. 6 start"


def write(name, vol, niter, workload):
    r = Oracle.from_volume(vol).solve(niter=niter, nls=5)
    out = {"source": SOURCE, "workload": workload, "niter": niter, "final_cost": float(r["cost"][-1]),
           "cost": [float(c) for c in r["cost"]]}
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["final_cost"])


def main(which):
    set_threads(os.cpu_count() or 1)  # the results do not depend on the thread count
    if which in ("all", "small"):
        write("small_oracle_cost.json", small_config(), 50,
              "synth.small_config(seed=1001): 64x64x16, 1 coil, echoes 0/2/10 ms, SNR 20 dB, beta 2^-3")
    if which in ("all", "full8"):
        write("full8_oracle_cost.json", full8_small_config(), 100,
              "synth.full8_small_config(seed=1007): 64x64x32, 8 coils, echoes 0/2/10 ms, +-250 Hz + 40 Hz step, "
              "SNR 15 dB, beta 2^-3")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "all")
