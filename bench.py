#!/usr/bin/env python
"""Benchmark of the hot path: circulation-based identification (Sec. 2.2.2,
Eq. 5) plus plain density-guided localization (Sec. 3.3.3, Eq. 6) of every
pierced plaquette, on a 512^3 complex64 random-wave tangle (16384 waves,
|k| in [0.15, 0.35] rad/h, 5% multiplicative amplitude noise; seeds 7 / 8).

One step = qtv_identify_localize over the whole field (identification sweep,
segment scan, and the pass that writes every pierced face and localizes it),
inputs resident in HBM (1 GiB field: larger than the 129 MB
L2, so no flush is needed).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl qtv|reference]

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(weak scaling; the path needs no data exchange), and the value is the total
grid points of all ranks over the slowest rank's time.  The reference arm
(--impl reference) times the FP64 CPU oracle on the host cores on a bounded
slab of the same field.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("grid points/s and HBM GB/s (identify+localize) vs peak; learned vs plain at "
          "≤0.05h")
UNIT = "grid points/s"
WORKLOAD = ("512^3 complex64 random-wave tangle: 16384 plane waves, |k| uniform in "
            "[0.15,0.35] rad/h, random directions, CN(0,1/W) amplitudes (seed 7), x (1+0.05 g) "
            "real multiplicative noise (seed 8); plain identify + localize")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["qtv", "reference"], default="qtv")
    p.add_argument("--n", type=int, default=512, help="grid edge (default 512)")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="host seconds of the oracle's timed CPU sample")
    p.add_argument("--cpu-planes", type=int, default=96,
                   help="planes of the field in the oracle's timed CPU sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--eager", action="store_true",
                   help="time K eager calls instead of one replay of their captured graph")
    p.add_argument("--soak", type=float, default=1.5,
                   help="seconds of untimed load before warm-up (clock sampling)")
    p.add_argument("--sweep-variant", type=int, default=-1,
                   help="identification sweep: 0 nibble, 1 bit-sliced, -1 library default")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the 16-snapshot batch against per-snapshot launches")
    p.add_argument("--no-learned", action="store_true",
                   help="skip training the learned locator and its report against plain")
    p.add_argument("--no-paper-size", action="store_true",
                   help="skip the identification + localization of a 2048^3 field")
    p.add_argument("--no-node-form", action="store_true",
                   help="skip the node-form, density-error, refinement, face-graph and line reports")
    return p.parse_args()


# DRAM bytes per node of the default (bit-sliced) sweep from one ncu capture,
# kept with the hash of the sweep sources it was taken on (profiles/, beside
# the capture's summary); valid while the sources hash to that value
SWEEP_SOURCES = ("paper_1911_12070_gb300/csrc/sweep_bits.cu",
                 "paper_1911_12070_gb300/csrc/sweep_common.cuh",
                 "paper_1911_12070_gb300/csrc/bits_layout.cuh")
TRAFFIC_FILE = "profiles/sweep_bits_traffic.json"


def sweep_sources_hash():
    import hashlib

    h = hashlib.sha256()
    for rel in SWEEP_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(variant):
    """(DRAM bytes per node, capture summary) of the bit-sliced sweep, or
    (None, reason) when the sweep timed is another kernel or has changed since
    the capture."""
    if variant == 0:
        return None, "nibble sweep: no current capture"
    path = os.path.join(ROOT, TRAFFIC_FILE)
    if not os.path.exists(path):
        return None, "no capture"
    with open(path) as fh:
        vals = json.load(fh)
    if vals.get("source_sha256") != sweep_sources_hash():
        return None, "kernel changed since the capture"
    return float(vals["traffic_bytes_per_node"]), vals.get("summary", TRAFFIC_FILE)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [r for t, r in self.rows if t0 <= t <= t1] or [r for _, r in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 4 + i and r[4 + i].lower().startswith("active")})
        pw = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


def field_pin(psi, n):
    """SHA-256 of the field's bytes and whether it equals the value pinned for
    this environment in synth/pins.json (the 512^3 workload only)."""
    from synth import make_pins

    sha = make_pins.sha256_of(psi)
    pinned = None
    if n == 512:
        try:
            pinned = make_pins.load()["device"].get(make_pins.environment_key(), {}).get(
                "512_waves_noise")
        except Exception:
            pinned = None
    return {"sha256": sha, "matches_pin": (sha == pinned) if pinned else None}


def make_field(n, device):
    import synth

    if n == 512:
        return synth.config_field("512_waves_noise", device=device)
    psi = synth.random_waves((n, n, n), synth.wave_spec(7, 16384 if n >= 512 else 4096),
                             device=device)
    return synth.multiplicative_noise(psi, 8)


def gain_report(q, noise):
    """RMS distance (h) to the clean plain cores of the plain solve of the
    noisy field and of the network on the noisy neighbourhoods, over all faces
    and over the tenth of the faces where the plain solve is worst."""
    import torch

    from paper_1911_12070_gb300 import learned

    clean, noisy = learned.field_pair(120, 256, 4096, noise, "cuda")
    test = learned.make_examples(q, clean, noisy)
    y = q.locator_forward(test["x"])
    xyz_n, _, _ = q.localize(noisy, test["ids"], test["w"])
    uvp = learned.face_uv(test["ids"], xyz_n, tuple(noisy.shape))
    ep = torch.sqrt(torch.sum((uvp - test["t"][:, :2]) ** 2, 1))
    el = torch.sqrt(torch.sum((y[:, :2] - test["t"][:, :2]) ** 2, 1))
    hard = ep > torch.quantile(ep, 0.9)
    rms = lambda e: float(torch.sqrt(torch.mean(e ** 2)))  # noqa: E731
    return {"faces": int(ep.numel()), "plain_rms_h": rms(ep), "network_rms_h": rms(el),
            "worst_decile_plain_rms_h": rms(ep[hard]),
            "worst_decile_network_rms_h": rms(el[hard])}


def learned_report(q, psi, ids, wnd, F, stream, reps=20):
    """Trains the learned locator (12 seeds of 256^3, about 2e6 faces, the
    library's own training kernels), then times plain localization and learned
    localization (dense layers on tcgen05, and on mma.sync for comparison) of
    the F faces of the bench field and measures the learned positions against
    the plain ones (the plain solve is the judge)."""
    import torch

    import paper_1911_12070_gb300 as qtv
    from paper_1911_12070_gb300 import learned

    torch.cuda.synchronize()
    t0 = time.time()
    losses = learned.fit(q)
    torch.cuda.synchronize()
    fit_s = time.time() - t0
    fid, w = ids[:F], wnd[:F]
    dev = psi.device
    outs = {}
    ms = {}
    for key, mode, path in (("plain", qtv.PLAIN, 0), ("mma", qtv.LEARNED, 0),
                            ("tcgen05", qtv.LEARNED, 1)):
        o = (torch.empty((F, 3), dtype=torch.float32, device=dev),
             torch.empty(F, dtype=torch.float32, device=dev),
             torch.empty(F, dtype=torch.uint8, device=dev))
        outs[key] = o
        q.locator_set_tensor_path(path)
        for _ in range(3):
            q.localize_into(psi, fid, w, *o, mode=mode, fallback_resid=1e-3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            q.localize_into(psi, fid, w, *o, mode=mode, fallback_resid=1e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[key] = e0.elapsed_time(e1) / reps
    q.locator_set_tensor_path(1 if ms["tcgen05"] < ms["mma"] else 0)
    # split of learned localization (library trace, tcgen05 path)
    q.trace_enable(True)
    q.trace_read(reset=True)
    q.locator_set_tensor_path(1)
    for _ in range(reps):
        q.localize_into(psi, fid, w, *outs["tcgen05"], mode=qtv.LEARNED, fallback_resid=1e-3)
    torch.cuda.synchronize()
    q.trace_enable(False)
    split = {k: v[1] / reps for k, v in q.trace_read(reset=True).items()
             if k in ("encode", "network", "head")}
    xyz_p, _, fl_p = outs["plain"]
    xyz_l, _, fl_l = outs["tcgen05"]
    good = (fl_p & qtv.FLAG_ANOMALOUS) == 0
    accepted = (fl_l & qtv.FLAG_LEARNED) != 0
    d2 = torch.sum((xyz_l - xyz_p) ** 2, 1)
    rms_all = float(torch.sqrt(torch.mean(d2[good])))
    rms_acc = float(torch.sqrt(torch.mean(d2[good & accepted])))
    flop = 2 * (128 * 256 + 256 * 256 + 256 * 3) * F
    # what the network gains over the plain solve (held-out field, seed 120):
    # at the training noise (5%) and with a second locator trained at 15%
    gain = {"against": "clean plain cores of a held-out 256^3 field (seed 120)",
            "noise_0.05": gain_report(q, 0.05)}
    q2 = qtv.Qtv(psi.device.index)
    try:
        learned.fit(q2, noise=0.15)
        gain["noise_0.15"] = gain_report(q2, 0.15)
    finally:
        q2.close()
    return {
        "gain": gain,
        "faces": F,
        "train": {"faces": "12 random-wave fields 256^3 (4096 waves, seeds 101-112), 5% noise "
                           "inputs, clean plain labels", "steps": int(len(losses)),
                  "seconds": fit_s, "final_loss": float(np.mean(losses[-50:]))},
        "plain_ms": ms["plain"], "learned_ms": ms["tcgen05"],
        "learned_mma_sync_ms": ms["mma"],
        "learned_split_ms": split,
        # network FLOPs over the network kernel's own time (the split), and
        # over the whole learned localization (encode + network + head)
        "learned_mlp_tflops": (flop / (split["network"] * 1e-3) / 1e12
                               if split.get("network") else None),
        "learned_localize_tflops": flop / (ms["tcgen05"] * 1e-3) / 1e12,
        "tensor_path": "tcgen05 (accumulators in tensor memory)",
        "accepted_frac": float(accepted.float().mean()),
        "rms_vs_plain_h": rms_all, "rms_vs_plain_accepted_h": rms_acc,
        "fallback_resid": 1e-3,
    }


def paper_size_report(peak, n=2048, waves=1024, reps=5):
    """Identification + plain localization of one field at the paper's own
    resolution, n^3 complex64 (2048^3: 64 GiB, the size of the paper's NLKG
    snapshots), on one GPU: CUDA-event time of `reps` steps after two warm-up
    steps, with a traced pass for the per-kernel times (the sweep against the
    HBM peak)."""
    import torch

    import paper_1911_12070_gb300 as qtv
    import synth

    nodes = n ** 3
    free, _ = torch.cuda.mem_get_info()
    need = 8 * nodes + 48 * 2 ** 30
    if free < need:
        return {"skipped": f"needs {need / 2 ** 30:.0f} GiB free, {free / 2 ** 30:.0f} GiB free"}
    t0 = time.time()
    psi = synth.random_waves((n, n, n), synth.wave_spec(2048, waves), device="cuda")
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    torch.cuda.empty_cache()  # the generator's temporaries
    h = qtv.Qtv(0)
    try:
        dev = psi.device
        cap = int(0.02 * nodes)
        h.reserve((n, n, n), cap)
        ids = torch.empty(cap, dtype=torch.int64, device=dev)
        wnd = torch.empty(cap, dtype=torch.int8, device=dev)
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        xyz = torch.empty((cap, 3), dtype=torch.float32, device=dev)
        resid = torch.empty(cap, dtype=torch.float32, device=dev)
        flags = torch.empty(cap, dtype=torch.uint8, device=dev)

        def step():
            h.identify_localize_into(psi, ids, wnd, count, xyz, resid, flags)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        F = int(count.item())
        if F < 0 or F > cap:
            return {"error": f"count {F} (capacity {cap})"}
        h.trace_enable(True)
        h.trace_read(reset=True)
        step()
        torch.cuda.synchronize()
        h.trace_enable(False)
        per_kernel = {k: v[1] / max(1, v[0]) for k, v in h.trace_read(reset=True).items()}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        step_bytes = 8 * nodes + 9 * F + F * (9 + 32 + 17)
        sweep_ms = per_kernel.get("sweep")
        out = {"grid": [n, n, n], "waves": waves, "field_gib": 8 * nodes / 2 ** 30,
               "pierced_faces": F, "ms_per_step": ms, "grid_points_per_s": nodes / (ms * 1e-3),
               "step_hbm_gbs": step_bytes / (ms * 1e-3) / 1e9,
               "kernels_ms": per_kernel, "generate_s": gen_s,
               "timing": f"CUDA events over {reps} eager steps after 2 warm-up steps; "
                         "kernels_ms from one traced step"}
        if sweep_ms:
            out["sweep_hbm_frac"] = 8 * nodes / (sweep_ms * 1e-3) / 1e9 / peak
        out["node_form"] = paper_size_node_form(h, psi, ids[:F], wnd[:F], peak)
        return out
    finally:
        h.close()
        del psi
        torch.cuda.empty_cache()


def paper_size_node_form(h, psi, fids, fw, peak, reps=3):
    """The node form (Sec. 2.2.2) of the paper-resolution field, from psi and
    from the face list: CUDA-event time per call after one warm-up call, and
    whether the two lists are equal."""
    import torch

    from paper_1911_12070_gb300 import QtvError

    dev = psi.device
    shape = tuple(psi.shape)
    nodes = psi.numel()
    try:
        cap = int(0.06 * nodes)
        n_ids = torch.empty(cap, dtype=torch.int64, device=dev)
        n_circ = torch.empty((cap, 3), dtype=torch.int8, device=dev)
        n_cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        f_ids = torch.empty(cap, dtype=torch.int64, device=dev)
        f_circ = torch.empty((cap, 3), dtype=torch.int8, device=dev)
        f_cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        f_tie = torch.zeros(1, dtype=torch.int32, device=dev)
        times = {}
        for name, call in (("from_psi", lambda: h.node_circulation_into(psi, n_ids, n_circ, n_cnt)),
                           ("from_faces", lambda: h.node_circulation_faces_into(
                               shape, fids, fw, f_ids, f_circ, f_cnt, f_tie))):
            call()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                call()
            e1.record()
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1) / reps
        nv, fn = int(n_cnt.item()), int(f_cnt.item())
        if nv > cap or fn > cap:
            return {"error": f"vortex nodes {max(nv, fn)} above capacity {cap}"}
        return {"vortex_nodes": nv, "ms_from_psi": times["from_psi"],
                "ms_from_faces": times["from_faces"], "tie": bool(int(f_tie.item())),
                "equal": bool(fn == nv and torch.equal(f_ids[:fn], n_ids[:nv])
                              and torch.equal(f_circ[:fn], n_circ[:nv])),
                "from_psi_hbm_frac": (8 * nodes + 11 * nv) / (times["from_psi"] * 1e-3) / 1e9 / peak}
    except QtvError as err:
        return {"error": str(err)}


def node_form_report(q, psi, xyz, count, stream, reps=20):
    """Node form of the circulation (Sec. 2.2.2: ring of 8 neighbours per node and
    plane, vortex node iff max |C| > pi) on the bench field, and the density error
    of Eq. 7 at the plain samples of the timed step (count read on the device)."""
    import torch

    from paper_1911_12070_gb300 import QtvError

    nodes = psi.numel()
    dev = psi.device
    cap = int(0.04 * nodes) + 1024
    ids = torch.empty(cap, dtype=torch.int64, device=dev)
    circ = torch.empty((cap, 3), dtype=torch.int8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    try:
        for _ in range(3):
            q.node_circulation_into(psi, ids, circ, cnt)
            q.density_error(psi, xyz, n_dev=count)
        torch.cuda.synchronize()
        nv = int(cnt.item())
        if nv > cap:
            return {"error": f"capacity {cap} below {nv} vortex nodes"}
        q.trace_enable(True)
        q.trace_read(reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            q.node_circulation_into(psi, ids, circ, cnt)
        e1.record(stream)
        torch.cuda.synchronize()
        tr = q.trace_read(reset=True)
        for _ in range(reps):
            e, mean_rho, rho_bar = q.density_error(psi, xyz, n_dev=count)
        tr_d = q.trace_read(reset=True)
        q.trace_enable(False)
    except QtvError as err:
        return {"error": str(err)}
    # the paper's graph over the vortex nodes (6-connectivity) and its components
    try:
        q.trace_enable(True)
        q.trace_read(reset=True)
        for _ in range(3):
            _, ndeg, ncmp, ncomp = q.node_graph(tuple(psi.shape), ids[:nv])
        trg = q.trace_read(reset=True)
        q.trace_enable(False)
        ngraph = {"ms": trg.get("graph", (1, 0.0))[1] / max(1, trg.get("graph", (1, 0.0))[0]),
                  "components": ncomp, "edges": int(ndeg.long().sum().item()) // 2}
    except QtvError as err:
        ngraph = {"error": str(err)}
    # the same node form from the identification's face list (a ring's
    # circulation is the sum of its four plaquettes' windings)
    try:
        fids, fw, _ = q.identify(psi)
        fcap = cap
        f_ids = torch.empty(fcap, dtype=torch.int64, device=dev)
        f_circ = torch.empty((fcap, 3), dtype=torch.int8, device=dev)
        f_cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        f_tie = torch.zeros(1, dtype=torch.int32, device=dev)
        shape = tuple(psi.shape)
        for _ in range(3):
            q.node_circulation_faces_into(shape, fids, fw, f_ids, f_circ, f_cnt, f_tie)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(reps):
            q.node_circulation_faces_into(shape, fids, fw, f_ids, f_circ, f_cnt, f_tie)
        f1.record(stream)
        torch.cuda.synchronize()
        fn = int(f_cnt.item())
        from_faces = {
            "ms_per_call": f0.elapsed_time(f1) / reps,
            "faces": int(fids.numel()),
            "tie": bool(int(f_tie.item())),
            "equal_to_psi_form": bool(fn == nv and torch.equal(f_ids[:fn], ids[:nv])
                                      and torch.equal(f_circ[:fn], circ[:nv])),
        }
    except QtvError as err:
        from_faces = {"error": str(err)}
    peak, peak_kind = peaks()
    kms = {k: v[1] / max(1, v[0]) for k, v in tr.items()}
    nf_ms = kms.get("node_form", 0.0)
    # algorithmic bytes: psi read once (8 B per node) + the vortex-node list
    # (8 B id + 3 B of windings per vortex node)
    alg = 8 * nodes + 11 * nv
    ach = alg / (nf_ms * 1e-3) / 1e9 if nf_ms > 0 else 0.0
    d_ms = tr_d.get("density", (1, 0.0))
    return {
        "ms_per_call": e0.elapsed_time(e1) / reps,
        "kernels_ms": kms,
        "vortex_nodes": nv,
        "vortex_node_fraction": nv / nodes,
        "roofline": {"bound": "hbm", "kernel": "node_form", "achieved": ach, "peak": peak,
                     "unit": "GB/s", "frac": ach / peak, "peak_source": peak_kind,
                     "algorithmic_bytes": alg},
        "vortex_node_graph": ngraph,
        "from_faces": from_faces,
        "density_error": {"e": e, "mean_abs_rho": mean_rho, "rho_bar": rho_bar,
                          "ms": d_ms[1] / max(1, d_ms[0]),
                          "points": "plain samples of the timed step"},
    }


def refine_report(q, psi, ids, count, F, stream, reps=5):
    """Sample refinement of Sec. 3.3.3 (descent of rho in the plane normal to the
    pseudo-vorticity) from the centres of the pierced faces of the timed step."""
    import torch

    from paper_1911_12070_gb300 import QtvError

    try:
        for _ in range(2):
            out = q.refine_samples(psi, face_ids=ids[:F], n_dev=count)
        torch.cuda.synchronize()
        q.trace_enable(True)
        q.trace_read(reset=True)
        for _ in range(reps):
            out = q.refine_samples(psi, face_ids=ids[:F], n_dev=count)
        tr = q.trace_read(reset=True)
        q.trace_enable(False)
        e_ref, _, _ = q.density_error(psi, out["xyz"], n_dev=count)
    except QtvError as err:
        return {"error": str(err)}
    fl = out["flags"]
    it = out["iters"].float()
    r = tr.get("refine", (1, 0.0))
    ms = r[1] / max(1, r[0])
    return {"ms": ms, "samples_per_s": F / (ms * 1e-3) if ms > 0 else None,
            "converged_fraction": (fl == 1).float().mean().item(),
            "no_tangent_fraction": ((fl & 2) != 0).float().mean().item(),
            "mean_steps": it.mean().item(), "max_steps": int(it.max().item()),
            "density_error_e": e_ref,
            "start": "centres of the pierced faces (one-cell estimates)"}


def graph_report(q, psi, ids, F, stream, reps=10):
    """Sample graph over the pierced faces of the timed step (faces sharing a unit
    cell, Sec. 3.1) and its connected components (Sec. 3.2)."""
    import torch

    from paper_1911_12070_gb300 import QtvError

    try:
        for _ in range(2):
            nbr, deg, comp, ncomp = q.face_graph(tuple(psi.shape), ids[:F])
        torch.cuda.synchronize()
        q.trace_enable(True)
        q.trace_read(reset=True)
        for _ in range(reps):
            nbr, deg, comp, ncomp = q.face_graph(tuple(psi.shape), ids[:F])
        tr = q.trace_read(reset=True)
        q.trace_enable(False)
    except QtvError as err:
        return {"error": str(err)}
    g = tr.get("graph", (1, 0.0))
    ms = g[1] / max(1, g[0])
    d = deg.long()
    sizes = torch.bincount(comp.long(), minlength=1)
    return {"ms": ms, "faces": F, "edges": int(d.sum().item()) // 2, "components": ncomp,
            "largest_component": int(sizes.max().item()),
            "branch_faces": int((d > 2).sum().item()),
            "faces_per_s": F / (ms * 1e-3) if ms > 0 else None}


def lines_report(q, psi, ids, wnd, xyz, F, stream, reps=5):
    """Vortex-core lines of the timed step's samples (Sec. 3.4): pieces of the face
    graph in walk order, oriented, and their Catmull-Rom curves."""
    import torch

    import paper_1911_12070_gb300 as qtv

    try:
        nbr, deg, comp, ncomp = q.face_graph(tuple(psi.shape), ids[:F])
        for _ in range(2):
            pieces, nodes = q.line_pieces(nbr, deg, comp, xyz[:F], ids[:F], wnd[:F])
            curve, first, length = q.piece_curves(xyz[:F], nodes, pieces, 8)
        torch.cuda.synchronize()
        q.trace_enable(True)
        q.trace_read(reset=True)
        for _ in range(reps):
            pieces, nodes = q.line_pieces(nbr, deg, comp, xyz[:F], ids[:F], wnd[:F])
            curve, first, length = q.piece_curves(xyz[:F], nodes, pieces, 8)
        tr = q.trace_read(reset=True)
        q.trace_enable(False)
    except qtv.QtvError as err:
        return {"error": str(err)}
    P = qtv.pieces_numpy(pieces)
    kms = {k: v[1] / max(1, v[0]) for k, v in tr.items()}
    types = np.bincount(P["comp_type"].astype(np.int64), minlength=4)
    # the rest of the vectorization: box means along the pieces (4 h), their
    # refinement in the plane normal to the pseudo-vorticity, and curves
    try:
        q.trace_enable(True)
        q.trace_read(reset=True)
        for _ in range(reps):
            means, tp = q.thin_pieces(xyz[:F], nodes, pieces, 4.0)
            ref = q.refine_samples(psi, xyz0=means)
            idn = torch.arange(means.shape[0], dtype=torch.int32, device=psi.device)
            rc_, rf_, rl_ = q.piece_curves(ref["xyz"], idn, tp, 8)
        tr2 = q.trace_read(reset=True)
        q.trace_enable(False)
        e_means, _, _ = q.density_error(psi, means)
        e_ref, _, _ = q.density_error(psi, ref["xyz"])
    except qtv.QtvError as err:
        return {"error": str(err)}
    k2 = {k: v[1] / max(1, v[0]) for k, v in tr2.items()}
    # the box-mean reduction of the whole face graph (lattice reading of Sec.
    # 3.3.2: clusters across branch points, passes to a fixed point), then the
    # refinement of its means and their Eq. 7 error
    try:
        for _ in range(2):
            lab, reps_, rmeans, rpasses = q.box_reduce(nbr, deg, xyz[:F], box=4.0)
        q.trace_enable(True, only="reduce")
        q.trace_read(reset=True)
        for _ in range(reps):
            lab, reps_, rmeans, rpasses = q.box_reduce(nbr, deg, xyz[:F], box=4.0)
        tr3 = q.trace_read(reset=True)
        q.trace_enable(False)
        rref = q.refine_samples(psi, xyz0=rmeans.float())
        e_rmeans, _, _ = q.density_error(psi, rmeans.float())
        e_rref, _, _ = q.density_error(psi, rref["xyz"])
        reduced = {"box_h": 4.0, "means": int(reps_.numel()), "passes": rpasses,
                   "ms": tr3["reduce"][1] / max(1, tr3["reduce"][0]),
                   "refined_converged_fraction": (rref["flags"] == 1).float().mean().item(),
                   "eq7_error_means": e_rmeans, "eq7_error_refined": e_rref}
    except qtv.QtvError as err:
        reduced = {"error": str(err)}
    return {"ms": kms, "pieces": int(len(P)), "closed_pieces": int(P["closed"].sum()),
            "box_reduced": reduced,
            "pieces_in_type_I_II_III": [int(types[1]), int(types[2]), int(types[3])],
            "reversed_pieces": int(P["reversed"].sum()), "curve_points": int(curve.shape[0]),
            "total_length_h": float(length.double().sum().item()),
            "thinned": {"box_h": 4.0, "means": int(means.shape[0]),
                        "ms": {"thin": k2.get("thin", 0.0), "refine": k2.get("refine", 0.0),
                               "curves": k2.get("curves", 0.0)},
                        "refined_converged_fraction": (ref["flags"] == 1).float().mean().item(),
                        "eq7_error_means": e_means, "eq7_error_refined": e_ref,
                        "total_length_h": float(rl_.double().sum().item())},
            "note": "line_pieces includes the host round trip of its count-only first call"}


def batch_report(q, stream, reps=10, learned=False):
    """The uneven 16-snapshot workload (8 x 256^3, 4 x 384^3, 3 x 512^3,
    1 x 768^3; seeds 201-216): one replay of the batch graph (persistent
    sweep over all snapshots, one finalize and one localization pass) against
    the same work as 16 separate qtv_identify_localize calls, identification
    plus plain localization in both; the learned-localization replay is timed
    too when a trained locator is loaded."""
    import torch

    import paper_1911_12070_gb300 as qtv
    import synth

    devs = synth.batch_fields("cuda")
    nodes = sum(d.numel() for d in devs)
    t0 = time.time()
    info = q.batch_plan(devs)
    plan_s = time.time() - t0
    dev = devs[0].device
    cap = int(info["faces"] * 1.02) + 1024
    ids = torch.empty(cap, dtype=torch.int64, device=dev)
    w = torch.empty(cap, dtype=torch.int8, device=dev)
    off = torch.zeros(len(devs) + 1, dtype=torch.int64, device=dev)
    xyz = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    resid = torch.empty(cap, dtype=torch.float32, device=dev)
    fl = torch.empty(cap, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    graph_ms = timed(lambda: q.batch_run_into(ids, w, off, xyz, resid, fl))
    faces = int(off[-1])
    # the same work as one call per snapshot
    o = off.cpu().numpy()
    per = []
    for i, d in enumerate(devs):
        m = int(o[i + 1] - o[i]) + 1024
        per.append((d, torch.empty(m, dtype=torch.int64, device=dev),
                    torch.empty(m, dtype=torch.int8, device=dev),
                    torch.zeros(1, dtype=torch.int64, device=dev),
                    torch.empty((m, 3), dtype=torch.float32, device=dev),
                    torch.empty(m, dtype=torch.float32, device=dev),
                    torch.empty(m, dtype=torch.uint8, device=dev)))
    q.reserve((768, 768, 768), max(int(o[i + 1] - o[i]) for i in range(len(devs))) + 1024)

    def singles():
        for d, a, b, c, x, r, f in per:
            q.identify_localize_into(d, a, b, c, x, r, f)

    single_ms = timed(singles)
    out = {
        "workload": "16 random-wave snapshots: 8 x 256^3, 4 x 384^3 (4096 waves), 3 x 512^3, "
                    "1 x 768^3 (16384 waves); seeds 201-216; identify + plain localize",
        "nodes": nodes, "faces": faces, "plan_seconds": plan_s,
        "tuned": {k: info[k] for k in ("warps_per_tile", "tile_columns", "ctas_per_sm", "zscale",
                                       "concurrent", "sweeps", "grid", "source", "candidates",
                                       "tuned_ms")},
        "graph_ms": graph_ms, "value": nodes / (graph_ms * 1e-3),
        "per_snapshot_ms": single_ms, "per_snapshot_value": nodes / (single_ms * 1e-3),
        "speedup_vs_per_snapshot": single_ms / graph_ms,
        "unit": UNIT,
        "hbm_gbs": (8 * nodes + 58 * faces) / (graph_ms * 1e-3) / 1e9,
    }
    if learned:
        out["learned_graph_ms"] = timed(lambda: q.batch_run_into(
            ids, w, off, xyz, resid, fl, mode=qtv.LEARNED, fallback_resid=1e-3))
    del devs, per
    q.batch_plan([torch.zeros((2, 2, 2), dtype=torch.complex64, device=dev)])  # release
    torch.cuda.empty_cache()
    return out


def oracle_sample(psi_host_slab, planes, want=False):
    """Oracle identify + localize on planes [0, planes) of a slab (with one halo
    plane); returns (seconds, nodes, faces[, (windings, flags)])."""
    import oracle

    t0 = time.perf_counter()
    w, fl = oracle.identify(psi_host_slab, k0=0, k1=planes)
    ids, wind = oracle.face_list(w)
    oracle.localize(psi_host_slab, ids, wind)
    dt = time.perf_counter() - t0
    nz, ny, nx = psi_host_slab.shape
    if want:
        return dt, planes * ny * nx, len(ids), (w, fl)
    return dt, planes * ny * nx, len(ids)


def sample_parity(w_or, fl_or, gpu_ids, gpu_w, shape, planes):
    """GPU windings against the oracle's on planes [0, planes): ambiguous faces
    (an edge within 1e-4 rad of +-pi) and how many of them, and of the others,
    differ."""
    import oracle

    nz, ny, nx = shape
    ids = np.asarray(gpu_ids, dtype=np.uint64)
    lin = (ids >> np.uint64(2)).astype(np.int64)
    sel = lin < planes * nx * ny
    g = np.zeros_like(w_or)
    o = (ids[sel] & np.uint64(3)).astype(np.int64)
    g[o, lin[sel] // (nx * ny), (lin[sel] // nx) % ny, lin[sel] % nx] = np.asarray(gpu_w)[sel]
    amb = (fl_or & oracle.AMBIGUOUS) != 0
    diff = g != w_or
    return {"planes": planes, "oracle_pierced": int(np.count_nonzero(w_or)),
            "oracle_ambiguous": int(amb.sum()),
            "ambiguous_differing": int(np.count_nonzero(diff & amb)),
            "unambiguous_differing": int(np.count_nonzero(diff & ~amb))}


def oracle_stage_baselines(psi, ids, wnd, xyz, F, planes=32, nref=50000):
    """The oracle's own rate on the stages beyond the step (host cores, bounded
    samples of the bench field): node form on the first `planes` z-planes,
    refinement from the first `nref` face centres, and the face graph with its
    components and the line pieces (classification, walk order, orientation)
    of the faces inside those planes."""
    import oracle
    from oracle import graph

    cores = oracle.max_threads()
    nz, ny, nx = psi.shape
    planes = max(2, min(planes, nz))
    slab = np.ascontiguousarray(psi[:planes].cpu().numpy())
    out = {}
    t = time.perf_counter()
    oracle.node_circulation(slab)
    dt = time.perf_counter() - t
    out["node_form"] = {"value": slab.size / dt, "unit": "nodes/s", "cores": cores,
                        "kind": "oracle",
                        "sample": f"{planes} z-planes ({slab.size} nodes), FP64, {dt:.2f} s"}
    idh = ids[:F].cpu().numpy().view(np.uint64)
    lin = (idh >> np.uint64(2)).astype(np.int64)
    kk = lin // (nx * ny)
    # refinement: face centres whose searches stay well inside the slab
    sel = np.flatnonzero(kk < planes - 4)[:nref]
    o = (idh[sel] & np.uint64(3)).astype(np.int64)
    ls = lin[sel]
    x0 = np.stack([ls % nx + 0.5 * ((o == 0) | (o == 2)),
                   (ls // nx) % ny + 0.5 * ((o == 0) | (o == 1)),
                   ls // (nx * ny) + 0.5 * ((o == 1) | (o == 2))], 1).astype(np.float64)
    t = time.perf_counter()
    oracle.refine(slab, x0)
    dt = time.perf_counter() - t
    out["refine"] = {"value": len(sel) / dt, "unit": "samples/s", "cores": cores,
                     "kind": "oracle",
                     "sample": f"{len(sel)} face centres of the first {planes - 4} planes, FP64, "
                               f"{dt:.2f} s"}
    # graph, components and lines: the faces that lie inside the slab
    inside = np.flatnonzero(kk < planes - 1)
    fid = idh[inside]
    fw = wnd[:F].cpu().numpy()[inside]
    fx = xyz[:F].cpu().numpy().astype(np.float64)[inside]
    t = time.perf_counter()
    g = graph.face_graph(fid, fw, fx, (planes, ny, nx))
    comps = graph.components(g)
    dt_graph = time.perf_counter() - t
    t = time.perf_counter()
    npieces = 0
    for c in comps:
        graph.classify(g, c)
        for _, path, closed in graph.ordered_lines(g, c):
            graph.orient(g, path, closed)
            npieces += 1
    dt_lines = time.perf_counter() - t
    out["face_graph"] = {"value": len(fid) / dt_graph, "unit": "faces/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"{len(fid)} faces of the first {planes - 1} planes, "
                                   f"{len(comps)} components, {dt_graph:.2f} s"}
    out["lines"] = {"value": len(fid) / dt_lines, "unit": "samples/s", "cores": 1,
                    "kind": "oracle",
                    "sample": f"the same faces: {npieces} pieces classified, ordered and "
                              f"oriented, {dt_lines:.2f} s"}
    return out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def slowest_ms(ms, device):
    """The largest of every rank's time (the job ends with its slowest rank)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, nodes_per_rank, steps, ms):
    """Whole-job grid points per second: all ranks' points over the slowest
    rank's time (each rank processes its own replica)."""
    return world_size * nodes_per_rank * steps / (ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth

    n = args.n
    planes = max(1, min(args.cpu_planes, n - 1))
    try:
        import torch

        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except Exception:
        dev = None
    # the slab [0, planes] of the same field (input preparation, untimed)
    spec = synth.wave_spec(7, 16384 if n >= 512 else 4096)
    if dev is not None:
        import torch

        z = synth.random_waves((n, n, n), spec, device=dev) if dev == "cuda" else None
        if z is not None:
            slab = synth.multiplicative_noise(z, 8)[: planes + 1].cpu().numpy()
            del z
            torch.cuda.empty_cache()
        else:
            slab = synth.multiplicative_noise(
                synth.random_waves_numpy((planes + 1, n, n), spec), 8)
    else:
        slab = synth.multiplicative_noise(synth.random_waves_numpy((planes + 1, n, n), spec), 8)
    slab = np.ascontiguousarray(slab)
    oracle.set_threads(cpu_cores())
    # size each step so that K steps take about a minute of host time
    dt1, _, _ = oracle_sample(slab[:2], 1)
    budget = 60.0 / max(1, args.steps)
    planes = int(max(1, min(planes, budget / max(dt1, 1e-6))))
    slab = np.ascontiguousarray(slab[: planes + 1])
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(slab, planes)
    times = []
    nodes = 0
    for _ in range(args.steps):
        dt, nodes, faces = oracle_sample(slab, planes)
        times.append(dt)
    total = sum(times)
    value = nodes * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"planes 0..{planes - 1}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"{planes} z-planes of the {n}^3 field ({nodes} nodes), "
                                   "FP64 identify + localize per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_qtv(args):
    import torch

    import paper_1911_12070_gb300 as qtv

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    qtv.build()
    q = qtv.Qtv(dev.index)
    q.configure_sweep(variant=args.sweep_variant)
    n = args.n
    psi = make_field(n, dev)
    torch.cuda.synchronize()
    nodes = n ** 3
    input_pin = field_pin(psi, n)
    stream = torch.cuda.current_stream()

    # size the outputs from one untimed call (with the statistics: ambiguous
    # faces of this field, which every step identifies alike)
    ids0, w0, id_stats = q.identify(psi, stats=True)
    F = ids0.numel()
    cap = int(F * 1.05) + 1024
    del ids0, w0
    q.reserve(tuple(psi.shape), cap)
    ids = torch.empty(cap, dtype=torch.int64, device=dev)
    wnd = torch.empty(cap, dtype=torch.int8, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    xyz = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    resid = torch.empty(cap, dtype=torch.float32, device=dev)
    flags = torch.empty(cap, dtype=torch.uint8, device=dev)

    def step():
        # identification + plain localization, fused (qtv_identify_localize)
        q.identify_localize_into(psi, ids, wnd, count, xyz, resid, flags)

    clk = ClockSampler(dev.index)
    clk.start()
    # soak (untimed) so the clock sampler sees the GPU under load
    t_end = time.time() + args.soak
    while time.time() < t_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # per-kernel times and launches per step from a traced pass (untimed: every
    # traced launch adds two events and their device gaps)
    q.trace_enable(True)
    q.trace_read(reset=True)
    for _ in range(10):
        step()
    torch.cuda.synchronize()
    q.trace_enable(False)
    per_kernel = q.trace_read(reset=True)
    launches_per_step = sum(v[0] for v in per_kernel.values()) / 10

    # the K timed steps as one CUDA graph (the calls allocate and synchronise
    # nothing), the sweep of every step bracketed by event-record nodes
    graph = torch.cuda.CUDAGraph()
    if args.eager:
        graph = None
    else:
        q.trace_enable(True, only="sweep")
        with torch.cuda.graph(graph):
            for _ in range(args.steps):
                step()
        q.trace_enable(False)
        graph.replay()  # upload (its steps are untimed warm-up)
        torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    if ws > 1:
        torch.distributed.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if graph is None:
        q.trace_enable(True, only="sweep")
        q.trace_read(reset=True)
    torch.cuda.synchronize()
    t0 = time.time()
    ev0.record(stream)
    if graph is None:
        for _ in range(args.steps):
            step()
    else:
        graph.replay()
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    q.trace_enable(False, only=None)
    trace = q.trace_read(reset=True)
    ms = ev0.elapsed_time(ev1)
    graphed = graph is not None
    del graph  # its event-record nodes hold events the handle reuses
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        ms = slowest_ms(ms, dev)
    F = int(count.item())
    clocks = clk.summary(t0 - 2.0, t1)

    # ---- end to end through the public API: every step copies the pinned host
    # field in and the packed samples and their count out
    # (qtv_identify_localize_host: two device copies of the field, so one
    # step's copy overlaps the previous step's identification)
    host_psi = torch.empty(psi.shape, dtype=torch.complex64, pin_memory=True)
    host_psi.copy_(psi)
    host_outs = [torch.empty(cap * 32, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    host_cnts = [torch.zeros(1, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    lib = qtv.lib()
    import ctypes

    grid = qtv.Grid.of(tuple(psi.shape))

    def e2e_step(i):
        rc = lib.qtv_identify_localize_host(q.h, ctypes.byref(grid),
                                            ctypes.c_void_p(host_psi.data_ptr()), cap,
                                            ctypes.c_void_p(host_outs[i % 2].data_ptr()),
                                            ctypes.c_void_p(host_cnts[i % 2].data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.qtv_last_error_string()

    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    ke = max(1, args.e2e_steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    c0 = time.perf_counter()
    for i in range(ke):
        e2e_step(i)
    enqueue_ms = (time.perf_counter() - c0) * 1e3 / ke
    e1.record(stream)
    torch.cuda.synchronize()
    assert all(int(c[0]) == F for c in host_cnts), "end-to-end sample count differs"
    d2h = ke * (cap * 32 + 8)
    ms_e2e = e0.elapsed_time(e1)
    if ws > 1:
        ms_e2e = slowest_ms(ms_e2e, dev)
    # the host link alone (outside every timed region): plain copies of the
    # pinned field to the device, the bound of the end-to-end rate
    link_dst = torch.empty_like(psi)
    with torch.cuda.stream(stream):
        link_dst.copy_(host_psi, non_blocking=True)
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for _ in range(5):
            link_dst.copy_(host_psi, non_blocking=True)
        l1.record(stream)
    torch.cuda.synchronize()
    link_gbs = 5 * 8 * nodes / (l0.elapsed_time(l1) * 1e-3) / 1e9
    del link_dst
    # and device-to-host copies of one step's packed samples alone (a
    # diagnostic: a failure here is reported, not raised)
    try:
        d2h_src = torch.empty(cap * 32, dtype=torch.uint8, device=psi.device)
        with torch.cuda.stream(stream):
            host_outs[0].copy_(d2h_src, non_blocking=True)
            d0 = torch.cuda.Event(enable_timing=True)
            d1 = torch.cuda.Event(enable_timing=True)
            d0.record(stream)
            for _ in range(5):
                host_outs[0].copy_(d2h_src, non_blocking=True)
            d1.record(stream)
        torch.cuda.synchronize()
        d2h_gbs = 5 * cap * 32 / (d0.elapsed_time(d1) * 1e-3) / 1e9
        del d2h_src
    except Exception as err:
        d2h_gbs = f"unmeasured: {err}"
    clk.stop()

    # ---- roofline of the dominant kernel (the sweep)
    peak, peak_kind = peaks()
    sweep_launches, sweep_ms = trace.get("sweep", (0, 0.0))
    sweep_avg_ms = sweep_ms / max(1, sweep_launches)
    # algorithmic bytes of one sweep: psi read once (8 B per node); halo rows,
    # tile overlaps, the per-warp tables and the staged records are overhead
    sweep_bytes = 8 * nodes
    achieved = sweep_bytes / (sweep_avg_ms * 1e-3) / 1e9 if sweep_avg_ms > 0 else 0.0
    traffic_per_node, traffic_src = profiled_traffic(args.sweep_variant)
    traffic = traffic_per_node * nodes if traffic_per_node is not None else None
    step_bytes = 8 * nodes + 9 * F + F * (9 + 32 + 17)
    ms_per_step = ms / args.steps
    launches = int(round(launches_per_step * args.steps))

    line = {
        "metric": METRIC,
        "value": job_value(ws, nodes, args.steps, ms),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [n, n, n], "pierced_faces": F,
                   "input_sha256": input_pin,
                   "l2": "inputs larger than L2 (1 GiB field, 129 MB L2); no flush",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "sweep", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "algorithmic_bytes": sweep_bytes,
                     "avg_ms": sweep_avg_ms},
        "step_hbm_gbs": step_bytes / (ms_per_step * 1e-3) / 1e9,
        "kernels_ms": {k: v[1] / max(1, v[0]) for k, v in per_kernel.items()},
        "kernels_ms_source": "10 traced eager steps outside the timed region",
        "timed_region": ("one replay of a CUDA graph of the K steps (sweeps bracketed by "
                         "event-record nodes)" if graphed else
                         "K eager steps (sweeps bracketed by events)"),
        "e2e": {"value": job_value(ws, nodes, ke, ms_e2e), "unit": UNIT,
                "h2d_bytes_per_step": 8 * nodes, "d2h_bytes_per_step": d2h // ke},
        "host_link": {"h2d_gbs": link_gbs,
                      "e2e_enqueue_ms_per_step": enqueue_ms,
                      "d2h_gbs": d2h_gbs,
                      "e2e_bound": link_gbs * 1e9 / 8 * ws,
                      "note": "pinned host-to-device copies of the field alone; the "
                              "end-to-end rate cannot exceed e2e_bound (grid points/s); "
                              "e2e_enqueue_ms_per_step is the host time to issue one "
                              "end-to-end step"},
        "gpu_launches": launches,
        "clocks": clocks,
        "ambiguous_faces": {"gpu": id_stats["ambiguous"], "pierced": id_stats["pierced"],
                            "source": "qtv_stats of an untimed identification of the same "
                                      "field (faces with an edge phase difference within "
                                      "1e-4 rad of +-pi)"},
    }

    if rank == 0 and not args.no_node_form:
        line["node_form"] = node_form_report(q, psi, xyz, count, stream)
        line["refine"] = refine_report(q, psi, ids, count, F, stream)
        line["face_graph"] = graph_report(q, psi, ids, F, stream)
        line["lines"] = lines_report(q, psi, ids, wnd, xyz, F, stream)

    if rank == 0 and not args.no_learned:
        line["learned"] = learned_report(q, psi, ids, wnd, F, stream)

    if rank == 0 and not args.no_batch:
        line["batch"] = batch_report(q, stream, learned=not args.no_learned)

    if rank == 0 and not args.no_paper_size:
        line["paper_resolution"] = paper_size_report(peak)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.no_node_form:
        import oracle

        oracle.set_threads(cpu_cores())
        for key, base in oracle_stage_baselines(psi, ids, wnd, xyz, F).items():
            if isinstance(line.get(key), dict):
                line[key]["cpu_baseline"] = base

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        planes = max(1, min(args.cpu_planes, n - 1))
        slab = np.ascontiguousarray(psi[: planes + 1].cpu().numpy())
        oracle.set_threads(cpu_cores())
        # repeat the slab until about args.cpu_seconds of host work
        dt, nn, reps = 0.0, 0, 0
        parity = None
        while reps < 1 or dt < args.cpu_seconds:
            if parity is None:
                d, m, _, (w_or, fl_or) = oracle_sample(slab, planes, want=True)
                nf = int(count.item())
                parity = sample_parity(w_or, fl_or, ids[:nf].cpu().numpy().view(np.uint64),
                                       wnd[:nf].cpu().numpy(), tuple(psi.shape), planes)
            else:
                d, m, _ = oracle_sample(slab, planes)
            dt += d
            nn += m
            reps += 1
        line["cpu_baseline"] = {
            "value": nn / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{planes} z-planes of the {n}^3 field ({nn // reps} nodes), FP64 identify "
                      f"+ localize, {reps} passes, {dt:.1f} s",
            "parity_on_sample": parity}
    if rank == 0:
        print(json.dumps(line), flush=True)
    q.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_qtv(args)


if __name__ == "__main__":
    sys.exit(main())
