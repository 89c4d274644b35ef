"""Autotuner of the grouped GEMM's CUDA-core tile shapes (run on the GPU).

Every CUDA-core tile shape of the grouped GEMM (64 x 64, 256 x 16, 128 x 32 and, for
FP32, 512 x 8) sums each output over k in the same order, so the choice changes the
speed only, never a result.  For every bucket of (element type, largest N, largest M)
this times one grouped launch of synthetic problems with each shape and keeps the
fastest; the table is written to gemm_tiles.json beside this file, which the binding
installs when it loads the library.  Launches on the tensor cores or on FP32 pairs are
not tuned.

    python -m paper_1602_01376_gb300.autotune [--quick]
"""
from __future__ import annotations

import json
import os
import sys

from . import GEMM_SHAPES, TILE_TABLE, iaskit_gemm_tile, iaskit_tune_gemm, load

# bucket b of N covers (8 << (b - 1), 8 << b]; of M (128 << (b - 1), 128 << b]
N_REP = [8, 16, 32, 64, 128, 256]
M_REP = [128, 256, 512, 1024, 2048]


def tune(quick: bool = False, reps: int = 5) -> dict:
    load()
    entries = []
    for fp64 in (1, 0):
        shapes = [s for s in GEMM_SHAPES if not (fp64 and s == "512x8")]
        for nb, n in enumerate(N_REP):
            for mb, m in enumerate(M_REP):
                if quick and (nb % 2 or mb % 2):
                    continue
                k = min(m, 512)                      # the contraction lengths of the method
                per = (m * k + k * n + m * n) * (8 if fp64 else 4)
                count = max(1, min(512, int(256e6 // per)))
                iaskit_gemm_tile(fp64, nb, mb, None)   # the bucket's entry is not used while timing
                ms = {s: iaskit_tune_gemm(fp64, m, n, k, count, s, reps) for s in shapes}
                best = min(ms, key=ms.get)
                entries.append({"fp64": fp64, "n_bucket": nb, "m_bucket": mb, "shape": best,
                                "M": m, "N": n, "K": k, "count": count,
                                "ms": {s: round(v, 4) for s, v in ms.items()}})
                print(json.dumps(entries[-1]), flush=True)
    return {"what": "fastest CUDA-core tile shape of one grouped GEMM launch per bucket "
                    "(identical results across shapes)", "entries": entries}


if __name__ == "__main__":
    table = tune(quick="--quick" in sys.argv)
    out = sys.argv[sys.argv.index("--out") + 1] if "--out" in sys.argv else TILE_TABLE
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    print(f"wrote {len(table['entries'])} entries to {out}")
