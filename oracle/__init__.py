"""FP64 CPU oracle for the stage-coupled implicit Runge-Kutta solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import anything
from this package.  The GPU library never calls it and shares no code with it:
the only module both sides use is ``workloads`` (seeded synthetic inputs, which
holds none of the method's arithmetic).

What it computes (Kirby & MacLachlan, "Extending Irksome"):

* ``tableaux``     Butcher tableaux: RadauIIA / Gauss-Legendre built by
                   collocation (App. A), and the printed ones (App. A, Sec. 2).
* ``fem``          Q1 mass and stiffness matrices, assembled cell by cell with
                   per-cell diffusivity (Sec. 2, eq. heat / rkheat).
* ``rk``           the Kronecker stage system (I (x) M + dt A (x) K) k = r of
                   Sec. 3, eq. block_struct_AI, solved by sparse LU, and the RK
                   update of Sec. 2.
* ``mg``           a sparse-matrix restatement of the geometric-multigrid
                   V-cycle used to approximate the diagonal blocks (Sec. 3.1).
* ``krylov``       FGMRES with the block preconditioners P_D / P_L / P_U
                   (Sec. 3.1, eq. pcbjac / pcbgs) for iteration-count parity.
* ``adjoint``      the discrete adjoint of the RK step and its gradient with
                   respect to per-cell log-diffusivity, plus a complex-step
                   derivative used to pin it.
* ``manufactured`` closed forms for the sine eigenmode used as pins.
"""
