"""Write the stored expected values that the GPU tests and the benchmark read.

Calls only the FP64 oracle (oracle/) on seeded synthetic inputs (synth/):
  small_oracle_cost.json  cost history of the 64x64x16 one-coil workload, 50 NCG-MLS-IC(0)
                          iterations (N_ls = 5): the target of the time-to-cost figure.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402
from synth import small_config  # noqa: E402


def main():
    vol = small_config()
    r = Oracle.from_volume(vol).solve(niter=50, nls=5)
    out = {"source": "FP64 oracle (oracle/fm_oracle.c), NCG-MLS-IC(0), N_ls = 5, from the Eq. 6 start",
           "workload": "synth.small_config(seed=1001): 64x64x16, 1 coil, echoes 0/2/10 ms, SNR 20 dB, beta 2^-3",
           "niter": 50, "final_cost": float(r["cost"][-1]), "cost": [float(c) for c in r["cost"]]}
    with open(os.path.join(HERE, "small_oracle_cost.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["final_cost"])


if __name__ == "__main__":
    main()
