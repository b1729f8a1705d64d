"""FP64 CPU oracle for the FAS multigrid Monge-Ampere solver.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports or links anything here.
"""
