"""FP64 CPU oracle of the TRD tracklet follower (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
import this package.  The CUDA library never uses it.
"""
