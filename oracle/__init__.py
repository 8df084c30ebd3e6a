"""Plain FP64 CPU oracle for (async-)Parareal on the heat equation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline / reference arm of ``bench.py`` use
it.  It shares no code with the CUDA path; the only common dependency is the
seeded input recipes in ``synthetic``.

Modules
-------
heat      the discrete operator A_kappa and the one-slice propagators F, G
          (explicit Euler, implicit Euler by Thomas or by CG), in FP64.
parareal  serial fine solve, synchronous Parareal (Algorithm 1, Eq. (11)),
          replay of an asynchronous event log (Eq. (12), Algorithm 2).
async_sim discrete-event simulation of asynchronous Parareal (Algorithm 2)
          on a virtual clock, producing event logs for the replay.
adjoint   discrete adjoint (reverse mode) of K synchronous iterations and of
          a logged asynchronous run.

Every function is slow and literal on purpose; each docstring names the
passage of the paper it follows.  Functions whose results no independent pin
fixes say "parity unpinned" in their docstring.
"""
