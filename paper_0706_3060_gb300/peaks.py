"""Measure the FP32 FFMA, packed FFMA2 and MUFU rsqrt throughput of the current GPU
with the library's own microbenchmark (nbody_peak_probe) and print one JSON line.

    python -m paper_0706_3060_gb300.peaks
"""
from __future__ import annotations

import ctypes
import json

from ._lib import check, load


def probe(kind: int, iters: int = 1 << 16) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    check(load().nbody_peak_probe(int(kind), int(iters), ctypes.byref(a), ctypes.byref(b)),
          "nbody_peak_probe")
    return a.value, b.value


def main() -> dict:
    import torch
    props = torch.cuda.get_device_properties(0)
    out = {"gpu": props.name, "sms": props.multi_processor_count}
    for kind, name, iters in ((0, "ffma", 1 << 16), (1, "ffma2", 1 << 16),
                              (2, "mufu_rsqrt", 1 << 16), (3, "ffma2_ffma_mix", 1 << 16),
                              (4, "grav_pair_loop_packed", 256), (5, "grav_pair_loop_scalar", 256)):
        per_clk, per_s = probe(kind, iters)
        out[name] = {"lane_ops_per_clk_per_sm": per_clk, "lane_ops_per_s": per_s}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
