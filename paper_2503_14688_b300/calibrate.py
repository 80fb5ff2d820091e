"""Sustained integer-instruction rates of this GPU (libisg_calib.so).

    python -m paper_2503_14688_b300.calibrate [--json out.json]

Prints, per operation class, operations per SM per clock at the SM clock
sampled during the run, and the Philox4x32-10 evaluations per SM per clock
(the quantity that bounds the sweep).
"""
import argparse
import ctypes
import json
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(PKG, "libisg_calib.so")

KINDS = {0: ("mul.wide (32x32->64) + xor", 8), 1: ("mul.hi + xor", 8), 2: ("mad.lo", 8),
         3: ("xor3", 8), 4: ("add3", 8), 5: ("philox4x32-10 call", 2),
         6: ("compare by sub.cc + addc", 8), 7: ("funnel shift", 8), 8: ("shift + or (C)", 8),
         9: ("add", 8), 10: ("byte permute", 8), 11: ("compare accumulated in C", 8),
         12: ("compare by borrow logic + funnel shift", 8),
         13: ("Ising word update, per site", 32), 14: ("sweep Philox call (folded)", 8),
         15: ("sweep Philox call, not unrolled", 8), 16: ("sweep Philox call, 4 per step", 4),
         17: ("sweep Philox call, 128 registers", 8), 18: ("Philox call unfolded, 8 unrolled", 8)}


def sm_clock_mhz():
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout
        return float(out.split()[0])
    except Exception:
        return None


def _load():
    from paper_2503_14688_b300 import build

    build.build_calib()
    lib = ctypes.CDLL(LIB)
    lib.isg_calib_run.restype = ctypes.c_float
    lib.isg_calib_run.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p]
    return lib


# The three rates the sweep's pipe-aware bound needs, as operations per SM
# per clock: the 32x32 -> 64 (high-half) multiply of Philox on the FMA-heavy
# pipe, a single-cycle logic op on the ALU pipe, a low-half multiply-add on
# the FMA-heavy pipe.
PIPE_KINDS = {"wide_multiply": 1, "alu_op": 7, "fma_op": 2}


def measure_rates(kinds=PIPE_KINDS, iters=20000):
    """Operations per SM per clock of each kind, on the current device.  The
    SM count comes from the device; the clock is the highest of two
    nvidia-smi samples taken around each timed launch (each about 0.25 s)."""
    import torch

    lib = _load()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.zeros(blocks, dtype=torch.int32, device="cuda")
    out = {"sms": sms}
    for name, kind in kinds.items():
        if lib.isg_calib_run(kind, blocks, threads, 100, sink.data_ptr()) < 0:  # warm-up
            raise RuntimeError("calibration kernel %d failed" % kind)
        mhz0 = sm_clock_mhz()
        ms = lib.isg_calib_run(kind, blocks, threads, iters, sink.data_ptr())
        mhz1 = sm_clock_mhz()
        if ms <= 0:
            raise RuntimeError("calibration kernel %d failed" % kind)
        mhz = max([m for m in (mhz0, mhz1) if m is not None] or [2032.0])
        ops = blocks * threads * iters * KINDS[kind][1]
        out[name] = {"per_sm_per_clk": ops / (ms * 1e-3) / sms / (mhz * 1e6), "sm_mhz": mhz,
                     "ms": ms}
    return out


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    lib = _load()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.zeros(blocks, dtype=torch.int32, device="cuda")
    res = {"sms": sms, "blocks": blocks, "threads": threads, "kinds": {}}
    for kind, (name, per_iter) in KINDS.items():
        iters = {5: 2000, 13: 400, 14: 400, 15: 400, 16: 400, 17: 400, 18: 400}.get(kind, 20000)
        lib.isg_calib_run(kind, blocks, threads, 100, sink.data_ptr())  # warm-up
        mhz0 = sm_clock_mhz()
        ms = lib.isg_calib_run(kind, blocks, threads, iters, sink.data_ptr())
        mhz1 = sm_clock_mhz()
        mhz = max(m for m in (mhz0, mhz1, 0.0) if m is not None) or 2032.0
        ops = blocks * threads * iters * per_iter
        per_sm_clk = ops / (ms * 1e-3) / sms / (mhz * 1e6)
        res["kinds"][name] = {"ms": ms, "ops": ops, "sm_mhz": mhz, "ops_per_sm_per_clk": per_sm_clk}
        print(f"{name:32s} {ms:9.2f} ms  {per_sm_clk:7.2f} /SM/clk  (SM {mhz:.0f} MHz)")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
