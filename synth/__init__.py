"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle."""
from .cube import (Scene, make_scene, workload_scene, WORKLOADS, batched_lines,  # noqa: F401
                   wavelengths, absorption_spectrum, background_model, plume_map)
