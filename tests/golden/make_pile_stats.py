"""Writes the FP64 oracle's pile statistics (repose angle and centre of mass), per
ensemble member and averaged, for the long-run statistical parity tests.  Calls only
the oracle.

  column (pile_column_32768.txt): scenes.pile_column, 32,768 spheres on a 24 x 24 x 57
      jittered lattice, seed 1001, mu = 0.2, dt = 5e-5 s, 20 projected-Jacobi
      iterations, 20,000 steps = 1 s, by which the pile has come to rest.
  pour (pour_pile_32768.txt): scenes.pour_pile, 32,768 spheres rained loosely onto a
      plane, seed 1005, mu = 0.6 (the column workload's friction), 20,000 steps = 1 s,
      by which the heap's slope has settled.

Members -1, 0, 1, 2 (the unperturbed scene and three one-ulp perturbations).

    python tests/golden/make_pile_stats.py [column|pour] [threads per run] [runs in parallel]
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

MEMBERS = (-1, 0, 1, 2)
CASES = {"column": ("pile_column", "pile_column_32768.txt", "mu=0.2"),
         "pour": ("pour_pile", "pour_pile_32768.txt", "mu=0.6")}


def run_member(args):
    case, member, threads = args
    import numpy as np
    import oracle
    from paper_2306_01369_gb300.stats import pile_statistics
    from paper_2306_01369_gb300 import scenes as S
    sc = getattr(S, CASES[case][0])(member)
    o = oracle.Sim(sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params, n_threads=threads)
    o.step(sc.n_steps)
    angle, com, nbins = pile_statistics(o.x, sc.mass, float(sc.pos_r[:, 3].max()))
    vmean = float(np.linalg.norm(o.v, axis=1).mean())
    return member, angle, com, nbins, vmean, float(sc.pos_r[:, 2].max())


def main():
    case = sys.argv[1] if len(sys.argv) > 1 else "column"
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count()
    par = int(sys.argv[3]) if len(sys.argv) > 3 else 1
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(par) as pool:
        res = pool.map(run_member, [(case, m, threads) for m in MEMBERS])
    import numpy as np
    angles = np.array([r[1] for r in res])
    coms = np.array([r[2] for r in res])
    fn, what = CASES[case][1], CASES[case][2]
    with open(os.path.join(HERE, fn), "w") as f:
        f.write(f"# FP64 oracle, scenes.{CASES[case][0]}(member), 32768 spheres, {what}, 20000 steps; "
                "written by make_pile_stats.py\n")
        for member, angle, com, nbins, vmean, h0 in res:
            f.write(f"# member {member}: angle_deg {angle:.6f} com {com[0]:.6e} {com[1]:.6e} {com[2]:.6e} "
                    f"fit_bins {nbins} mean_speed {vmean:.3e}\n")
        f.write(f"members: {len(res)}\n")
        f.write(f"angle_deg: {angles.mean():.6f}\n")
        f.write(f"com: {coms[:, 0].mean():.9e} {coms[:, 1].mean():.9e} {coms[:, 2].mean():.9e}\n")
        f.write(f"h0: {res[0][5]:.9e}\n")


if __name__ == "__main__":
    main()
