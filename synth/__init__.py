"""Seeded synthetic inputs (velocity models, geometry, records) shared by the
CPU oracle tests and the CUDA path.  Holds no wave-equation arithmetic."""
from .workloads import (Workload, WORKLOADS, small2d, thrust2d, salt2d, arid2d, layered3d,
                        tiny2d, tiny3d, true_model, initial_model, sample_models,
                        random_records, add_noise)
from . import models
