"""Write tests/golden/config_oracle_costs.json: the FP64 oracle's Qfactor
(Alg. 1, with the reset of Sec. III-A2 every 40 sweeps) on the two smallest
seeded workloads, run to dist_tol = 1e-10 or 500 sweeps:

  3q_6gates    3 qubits, 6 U(4) gates alternating on (0,1), (1,2), a target
               reachable from seeded Haar gates (seed 2024), start 0;
  6q_30gates   6 qubits, linear brickwork of 12 layers (30 U(4) gates),
               starts 0 and 1 of the seeded problem (seed 2024), on the
               reachable target and on a Haar-random 64 x 64 target
               (haar_unitary(64, rng(2024))).

Each start runs alone (starts are independent; the lock-step multistart rule
only decides when a run stops, and no start here stops before 500 sweeps
except by reaching dist_tol).  The GPU runs the same inputs in
tests/test_gpu_configs.py and bench.py reports both side by side.

Only the oracle computes these values.  Usage: python tests/golden/make_config_costs.py
(about a minute on 8 cores).
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as orc  # noqa: E402
import qf_inputs as qi  # noqa: E402

SEED = 2024
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config_oracle_costs.json")


def config_inputs():
    """The seeded inputs of both workloads (shared with the GPU test)."""
    locs3 = np.array([[0, 1], [1, 2]] * 3, dtype=np.int32)
    inst3 = qi.make_problem(3, locs3, 1, seed=SEED)
    locs6 = qi.brickwork_locations(6, 12)
    inst6 = qi.make_problem(6, locs6, 16, seed=SEED)
    haar6 = qi.haar_unitary(64, qi.rng(SEED))
    return inst3, inst6, haar6


def run(V, start, locs, n):
    r = orc.qfactor(V, start, locs, n, orc.QFactorOptions(dist_tol=1e-10, max_iter=500, reset_iter=40))
    return {"cost": float(r["cost"]), "sweeps": int(r["sweeps"]), "reason": r["reason"]}


def main():
    inst3, inst6, haar6 = config_inputs()
    out = {
        "about": "FP64 oracle (oracle/qfactor_oracle.py, Alg. 1 Qfactor with reset_iter 40) on the "
                 "seeded 3- and 6-qubit workloads; written by tests/golden/make_config_costs.py",
        "dist_tol": 1e-10, "max_sweeps": 500, "reset_iter": 40,
        "3q_6gates": {"start0": run(orc.circuit_unitary(inst3.target_gates, inst3.locs, 3),
                                    inst3.starts[0], inst3.locs, 3)},
        "6q_30gates": {},
    }
    V6 = orc.circuit_unitary(inst6.target_gates, inst6.locs, 6)
    for tname, V in (("reachable", V6), ("haar", haar6)):
        out["6q_30gates"][tname] = {f"start{s}": run(V, inst6.starts[s], inst6.locs, 6) for s in (0, 1)}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
