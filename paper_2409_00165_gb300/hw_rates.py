"""Hardware rates of the current GPU that this library's kernels are measured against:
FP64 FMA, MUFU tanh, tcgen05.mma by N and A-operand source, L2 -> shared-memory bulk
copies (see fos_measure_hw_rates in include/fos.h).

    python -m paper_2409_00165_gb300.hw_rates
"""
from __future__ import annotations

import json


def main() -> None:
    from . import fos
    print(json.dumps(fos.fos_measure_hw_rates()))


if __name__ == "__main__":
    main()
