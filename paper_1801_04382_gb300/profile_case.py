"""Small profiling case of the interval kernels (for ncu captures that must stay small).

    python -m paper_1801_04382_gb300.profile_case [fp32|fp64] [M] [tile_traj]

Four-node cascaded chain (d = 6561, dt = 0.01), M trajectories (default 304 = two CTAs per
SM of work), 12 intervals: guess sweep, backward sweep, updating forward sweep, with the
library's per-launch event profiling printed at the end.  A few hundred MB on the device.
"""
import sys

import numpy as np

import synth_inputs as si
from paper_1801_04382_gb300 import Problem, cascaded_chain


def main(argv):
    prec = argv[1] if len(argv) > 1 else "fp32"
    M = int(argv[2]) if len(argv) > 2 else 304
    tile = int(argv[3]) if len(argv) > 3 else 0
    nt, T = 12, 0.12
    net = cascaded_chain(4, 2)
    eps0 = si.guess_pulses(4, nt, T, 1.0)
    S = si.shape_functions(4, nt, T)
    lam = np.full(4, 10.0)
    U = si.uniforms(4, 4, M, 25)
    with Problem(net, T, nt, M, eps0, S, lam, U, precision=prec, tile_traj=tile) as p:
        info = p.info
        print(f"d={info.d} tile_traj={info.tile_traj} threads={info.threads} cheb_terms={info.cheb_terms} "
              f"tiles={info.n_tiles}")
        p.forward(False)
        p.set_profiling(True)
        p.backward()
        p.forward(True)
        prof = p.profile()
        for k, (ms, n) in prof.items():
            print(f"{k}_kernel: {n} launches, {ms:.3f} ms, {ms / max(n, 1):.4f} ms/launch")


if __name__ == "__main__":
    main(sys.argv)
