"""FP64 CPU oracle of the sparse albedo-corrected matched filter.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.
"""
from .mf_oracle import *  # noqa: F401,F403
from .mf_oracle import (ALBEDO, SPARSE, LITERAL, PENALTY_NO_ALBEDO, NotSPD,  # noqa: F401
                        retrieve, retrieve_partition, partitions, valid_pixels,
                        mean_vector, covariance_about, albedo_factor,
                        amplification, retrieve_amplification, partition_energy,
                        retrieve_energy)
from .mf_grad import retrieve_partition_t, vjp as grad_vjp  # noqa: F401,E402
