"""FP64 CPU oracle for trajectory-parallel Krotov optimisation (Goerz & Jacobs, arXiv:1801.04382).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` may import it.
The product path (``paper_1801_04382_gb300``) never imports, links or executes it, and the
oracle imports nothing from the product: the two share no code.  Both are fed from the seeded
input generators of ``synth_inputs`` only.

It is a plain, slow, obviously correct restatement of the method:

* ``model``     dense operators by explicit Kronecker products (Sec. 3.1, Eqs. ham, ham_interaction).
* ``propagate`` exact per-interval propagators: dense expm, and an FP64 Chebyshev series
                for large d pinned against expm (Sec. 2.1 / 2.2, piecewise-constant controls).
* ``mcwf``      MCWF trajectories with bisected jump times (Sec. 2.1), the trajectory
                functional (Eq. functional_traj), the pathwise backward co-state sweep and the
                sequential independent-trajectory Krotov update (Eq. independent_traj_update),
                Krotov's functional (Eq. krotov_functional).
* ``gradient``  exact frozen-record gradient and finite differences (Eq. gradient, Sec. 2.2).
* ``lindblad``  density-matrix reference (Eqs. lindblad, rho_traj_expansion).

Parity status of each function (what pins it) is listed in the tests under ``tests/``.
"""
from . import model, propagate, mcwf, gradient, lindblad  # noqa: F401
