"""Seeded synthetic inputs shared by the FP64 oracle, the CUDA library's tests and the benchmark.

This package only *produces inputs*: detector site geometry, the analytic PSD, coloured Gaussian
noise, injected signals following the paper's data model (the H1 hypothesis x = h + n of Sec. II
and the detector response of eq. detresponse), particle batches and workload descriptions.
It computes no part of the coherent fitness (no correlation, no FFT over t_c, no antenna
projection, no argmax) and imports neither ``oracle`` nor the CUDA package.
"""

from .sites import SITES, detector_geometry
from .psd import aligo_fit_psd, psd_on_grid
from .workloads import (Workload, SMALL, C1, C2, PAPER_DNS, PAPER_TAU_BOX, workload_by_name, make_dataset,
                        make_particles, chirp_time_box)

__all__ = [
    "SITES", "detector_geometry", "aligo_fit_psd", "psd_on_grid",
    "Workload", "SMALL", "C1", "C2", "PAPER_DNS", "PAPER_TAU_BOX", "workload_by_name", "make_dataset",
    "make_particles", "chirp_time_box",
]
