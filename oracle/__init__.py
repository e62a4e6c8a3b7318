"""FP64 CPU oracle of FRAM (arXiv 2508.00887).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg to check and time the CUDA path.  The product
package never imports it, and it imports nothing from the product package.
"""
from .fram_oracle import (DEFAULTS, DegenerateError, FRAResult, FramResult, InvalidInputError,
                          SDSNResult, accuracy, damped_update, fra_exact, fra_residual, fram,
                          gamma, simplex_thresholds, gradient, gradient_columns,
                          initial_assignment,
                          lap_max, matching_error, node_affinity, objective, p1, p2, p3,
                          prescale, sdsn, validate)

__all__ = ["DEFAULTS", "DegenerateError", "FRAResult", "fra_exact", "fra_residual",
           "simplex_thresholds", "FramResult", "InvalidInputError", "SDSNResult",
           "accuracy", "damped_update", "fram", "gamma", "gradient", "gradient_columns",
           "initial_assignment",
           "lap_max", "matching_error", "node_affinity", "objective", "p1", "p2", "p3", "prescale", "sdsn",
           "validate"]
