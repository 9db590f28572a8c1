"""Writes the full-size golden records tests/golden/fullsize_<name>.json.

Each record holds what the CPU oracle (oracle/, the plain restatement of the
paper's Sec. 3-4) computes for one full-size workload: SHA-256 digests of the
inputs f and fhat (so a run elsewhere can prove it regenerated the same
bits), of the edit list (indices as little-endian uint32, values as the raw
bytes of the field's type), of both label arrays (int32), the status, the
edit count and every counter of the fix. The inputs come from
paper_2406_09423_gb300.synth, whose generators give the same bits on every
machine; nothing here calls the CUDA library.

Usage: python tests/golden/make_fullsize.py NAME [NAME ...]   (see CONFIGS)
One oracle fix at 512^3 runs for hours on one core; run the names as
separate processes to use several cores.
"""
from __future__ import annotations

import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# name -> (generator call, description, relative bound xi / range)
CONFIGS = {
    "lognormal256_1e-3": ("lognormal3d(256, 1)", "3D 256^3 float32 lognormal, P(k) ~ k^-3, seed 1", 1e-3),
    "lognormal256_1e-4": ("lognormal3d(256, 1)", "3D 256^3 float32 lognormal, P(k) ~ k^-3, seed 1", 1e-4),
    "ocean_1e-3": ("ocean2d(3600, 2400, 2)", "2D 3600x2400 float32 ocean (gradient + 400 eddies + noise), seed 2", 1e-3),
    "ocean_1e-4": ("ocean2d(3600, 2400, 2)", "2D 3600x2400 float32 ocean (gradient + 400 eddies + noise), seed 2", 1e-4),
    "ocean_1e-5": ("ocean2d(3600, 2400, 2)", "2D 3600x2400 float32 ocean (gradient + 400 eddies + noise), seed 2", 1e-5),
    "turb512_1e-3": ("turbulence3d(512, 3)", "3D 512^3 float32 turbulence (256 modes, Kolmogorov), seed 3", 1e-3),
    "turb512_1e-4": ("turbulence3d(512, 3)", "3D 512^3 float32 turbulence (256 modes, Kolmogorov), seed 3", 1e-4),
    "turb512_1e-5": ("turbulence3d(512, 3)", "3D 512^3 float32 turbulence (256 modes, Kolmogorov), seed 3", 1e-5),
}


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make(name: str) -> dict:
    import oracle
    from paper_2406_09423_gb300 import synth

    call, desc, rel = CONFIGS[name]
    t0 = time.time()
    f = eval("synth." + call, {"synth": synth})
    xi = synth.xi_for(f, rel)
    fhat = synth.quantise(f, xi)
    t1 = time.time()
    r = oracle.fix(f, fhat, xi)
    t2 = time.time()
    return {
        "name": name,
        "generator": "synth." + call,
        "workload": desc,
        "rel": rel,
        "xi": xi,
        "shape": list(f.shape),
        "dtype": str(f.dtype),
        "status": int(r.status),
        "n_edits": int(r.edit_idx.size),
        "counts": r.counts,
        "sha256": {
            "f": digest(f),
            "fhat": digest(fhat),
            "edit_idx": digest(r.edit_idx.astype("<u4")),
            "edit_val": digest(r.edit_val),
            "label_max": digest(r.label_max.astype("<i4")),
            "label_min": digest(r.label_min.astype("<i4")),
        },
        "oracle_seconds": round(t2 - t1, 1),
        "generate_seconds": round(t1 - t0, 1),
        "host": f"{platform.machine()} {platform.processor() or ''}".strip(),
    }


def main(argv):
    names = argv or sorted(CONFIGS)
    for name in names:
        rec = make(name)
        path = os.path.join(HERE, f"fullsize_{name}.json")
        with open(path + ".tmp", "w") as fh:
            json.dump(rec, fh, indent=1)
            fh.write("\n")
        os.replace(path + ".tmp", path)
        print(name, rec["status"], rec["n_edits"], rec["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
