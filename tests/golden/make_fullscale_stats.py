"""Write ``fullscale_stats.json``: the within-population statistics of the
full microcircuit (scale 1, 77,169 neurons) simulated by the CPU oracle with
several network/background seeds, for the statistical comparison the paper
makes between simulators past the divergence horizon (Sec. 4.2: rates, CV of
ISI and correlations of binned spike trains, the first 1 s discarded,
Sec. 2.1).

Calls only ``oracle/`` and the seeded inputs of ``workload/``.  Each seed runs
in its own process (the oracle's step loop is single-threaded).  Run from the
repository root:

    python tests/golden/make_fullscale_stats.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SEEDS = [202, 303, 404, 505]
STEPS = 30000            # 3 s biological at dt = 0.1 ms
DISCARD = 10000          # the first 1 s (Sec. 2.1)


def one(seed):
    import oracle
    import workload
    t0 = time.time()
    cfg = workload.microcircuit(1.0, seed=seed)
    net = oracle.Network(cfg, n_threads=max(1, (os.cpu_count() or 4) // len(SEEDS)))
    sim = oracle.Simulation(net)
    sim.run(STEPS)
    st, ids = sim.raster()
    stats = oracle.population_statistics(cfg, st, ids, DISCARD, STEPS)
    stats["seed"] = seed
    stats["events"] = sim.counters()["events"]
    stats["spikes"] = int(st.size)
    stats["seconds"] = time.time() - t0
    return stats


def main():
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        runs = pool.map(one, SEEDS)
    out = {"_source": "CPU oracle (oracle/), full microcircuit at scale 1 (workload.microcircuit"
                      "(1.0, seed)); statistics of Sec. 4.2 over steps [%d, %d)" % (DISCARD, STEPS),
           "_script": "tests/golden/make_fullscale_stats.py",
           "steps": STEPS, "discard": DISCARD, "runs": runs}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullscale_stats.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
