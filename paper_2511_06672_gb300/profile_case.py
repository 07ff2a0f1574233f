"""Run one seeded benchmark circuit through libgcamps (for profiling one engine launch).

    python -m paper_2511_06672_gb300.profile_case --d 3 --n 12 --layers 10 --t 12 --chi 64 --seed 1 --repeat 2

Each repetition resets the simulator and runs the whole gate list in one engine launch.
"""
import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--n", type=int, default=12)
    ap.add_argument("--layers", type=int, default=10)
    ap.add_argument("--t", type=int, default=12)
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--cutoff", type=float, default=1e-12)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args()
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import numpy as np
    import paper_2511_06672_gb300 as G
    from synth import brickwork_circuit
    ops, begin = [], [0]
    for b in range(a.batch):
        o = G.ops_from_gates(brickwork_circuit(a.n, a.d, a.layers, a.t, a.seed + b), a.d)
        ops.append(o)
        begin.append(begin[-1] + len(o))
    ops = np.concatenate(ops)
    sim = G.Simulator(a.n, a.d, chi_max=a.chi, cutoff=a.cutoff, batch=a.batch)
    for r in range(a.repeat):
        sim.reset()
        t0 = time.perf_counter()
        sim.run(ops, np.array(begin, dtype=np.int32))
        sim.sync()
        st = sim.stats()
        print(f"rep {r}: {time.perf_counter() - t0:.4f} s  T={st['t_gates']} cands={st['candidates_scored']} "
              f"max_chi={st['max_chi']} flops={st['scoring_flops']:.3e}", flush=True)
    sim.close()


if __name__ == "__main__":
    main()
