"""Write ``microcircuit_table.json``: the seeded synthetic connection table.

Run from the repository root:  python -m workload.make_table
The table is an input of the simulation, not an expected value; it is drawn
by :func:`workload.generate_connection_table` (seed 1909) and stored so that
every run, on every machine, uses the same numbers.
"""
import json
import os

import workload


def main():
    p = workload.generate_connection_table(1909)
    out = {
        "description": "synthetic stand-in for the 8x8 connection-probability table "
                       "(p[target][source]); see workload.generate_connection_table",
        "seed": 1909,
        "conn_prob": [[float(v) for v in row] for row in p],
        "k_ext": workload.background_indegrees(),
        "u0_lo": 0.0,
        "u0_hi": 15.0,
    }
    path = os.path.join(os.path.dirname(__file__), "microcircuit_table.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
