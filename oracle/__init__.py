"""CPU oracle for hashed path space filtering: test infrastructure only.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package; the CUDA library never does."""
