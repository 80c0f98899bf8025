"""ORQA oracle package -- TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU
baseline leg of the benchmark).  The CUDA library never imports it."""
from .oracle import (Oracle, build, run_layers, index_from_codes, index_from_label,
                     codes_from_index, gate_index, phase_exponent, rotation_cos_sin, histogram)

__all__ = ["Oracle", "build", "run_layers", "index_from_codes", "index_from_label",
           "codes_from_index", "gate_index", "phase_exponent", "rotation_cos_sin", "histogram"]
