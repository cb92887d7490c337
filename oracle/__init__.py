"""FP64 CPU oracle for the OMM hot path: TEST INFRASTRUCTURE ONLY.

Only the tests, the package's smoke check and the benchmark's CPU-baseline arm
import this package.  The CUDA library never does, and shares no code with it.
"""
