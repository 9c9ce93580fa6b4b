"""FP64 CPU oracle of the coherent fitness and of the lbest PSO step (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline / reference arm use this package.
The CUDA library never imports, links or calls it.
"""
