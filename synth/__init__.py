"""Seeded synthetic inputs for the TRD tracklet follower.

This package is the only code that the FP64 oracle and the CUDA library
share: it draws truth tracks and turns them into seeds and tracklets.  It
simulates the detector with its own global-helix arithmetic and holds none
of the follower's arithmetic (no local-frame transport, no covariance
algebra, no chi2, no Kalman update).
"""
from .timeframe import (  # noqa: F401
    Timeframe,
    make_timeframe,
    make_workload,
    WORKLOADS,
    efficiency_purity,
)
