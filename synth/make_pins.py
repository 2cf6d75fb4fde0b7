"""Writes synth/pins.json: the SHA-256 of the bytes of every seeded field the
tests and the benchmark use, so that a change of the inputs (a new generator,
a new BLAS or cuBLAS) is detected instead of silently moving every parity
case and benchmark number.

Host fields (numpy, FP64 evaluation rounded once to complex64) are pinned
once.  Device fields (torch on a GPU: FP64 phase tables, each z-plane a
complex64 GEMM accumulated in FP32 by the library that torch calls) depend
on that library, so their hashes are keyed by the environment that made them
(torch version, CUDA version, GPU name); other environments are not pinned.

    python -m synth.make_pins            # host fields (no GPU needed)
    python -m synth.make_pins --device   # also the device fields (on a GPU)

Calls only synth (no method arithmetic is involved).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
PINS = os.path.join(HERE, "pins.json")


def sha256_of(a) -> str:
    """SHA-256 of the raw bytes of a complex64 array or tensor (C order)."""
    if not isinstance(a, np.ndarray):
        a = a.contiguous().cpu().numpy()
    assert a.dtype == np.complex64
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def host_fields():
    """name -> zero-argument maker of every host field that is pinned."""
    return {
        "64_analytic": lambda: synth.analytic_line_ring(),
        "64_analytic_line_only": lambda: synth.analytic_line_ring(with_ring=False),
        "waves_24x40x130_seed1_256": lambda: synth.random_waves_numpy(
            (24, 40, 130), synth.wave_spec(1, 256)),
        "waves_33x45x67_seed3_512": lambda: synth.random_waves_numpy(
            (33, 45, 67), synth.wave_spec(3, 512)),
    }


def device_fields(device="cuda"):
    """name -> maker of every device field that is pinned (per environment)."""
    out = {
        "256_waves_seed1": lambda: synth.config_field("256_waves", device=device, seed=1),
        "256_waves_seed2": lambda: synth.config_field("256_waves", device=device, seed=2),
        "512_waves_noise": lambda: synth.config_field("512_waves_noise", device=device),
    }
    for i, (n, w) in enumerate(synth.BATCH16):
        out[f"batch16_{i:02d}_{n}_seed{201 + i}"] = (
            lambda n=n, w=w, i=i: synth.random_waves((n, n, n), synth.wave_spec(201 + i, w),
                                                     device=device))
    return out


def environment_key() -> str:
    import torch

    return (f"torch {torch.__version__} cuda {torch.version.cuda} "
            f"{torch.cuda.get_device_name(0)}")


def load():
    if not os.path.exists(PINS):
        return {"host": {}, "device": {}}
    with open(PINS) as fh:
        return json.load(fh)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--device", action="store_true", help="also pin the device fields")
    ap.add_argument("--out", default=PINS)
    args = ap.parse_args()
    pins = load()
    pins["host"] = {k: sha256_of(f()) for k, f in host_fields().items()}
    if args.device:
        import torch

        env = environment_key()
        d = {}
        for k, f in device_fields().items():
            t = f()
            d[k] = sha256_of(t)
            del t
            torch.cuda.empty_cache()
        pins.setdefault("device", {})[env] = d
    with open(args.out, "w") as fh:
        json.dump(pins, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
