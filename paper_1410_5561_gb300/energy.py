"""GPU energy per lattice-site update from NVML's total-energy counter (read only).

Section IV of the paper measures energy per LUP of the blocked and plain schemes from the
CPU's RAPL counters and relates it to the code balance (Eq. 1: energy grows with the data
moved). The GPU counterpart read here is NVML's cumulative board energy of the device
(millijoules since the driver loaded); it cannot separate DRAM from core energy, so the
figure is the whole board's. Nothing is ever set through NVML: the meter opens the library,
finds the device by UUID, reads the counter and closes the library.

``nvml`` may be any object with the four calls used below (a fake in the CPU tests); by
default the system's ``libnvidia-ml.so.1`` is opened with ctypes.
"""
from __future__ import annotations

import ctypes
import time


class _NvmlLib:
    """The few NVML entry points used, through ctypes (0 = NVML_SUCCESS)."""

    def __init__(self):
        self.L = ctypes.CDLL("libnvidia-ml.so.1")
        self.L.nvmlDeviceGetHandleByUUID.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
        self.L.nvmlDeviceGetTotalEnergyConsumption.argtypes = [ctypes.c_void_p,
                                                               ctypes.POINTER(ctypes.c_ulonglong)]

    def init(self) -> int:
        return self.L.nvmlInit_v2()

    def shutdown(self) -> int:
        return self.L.nvmlShutdown()

    def handle_by_uuid(self, uuid: str):
        h = ctypes.c_void_p()
        rc = self.L.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h))
        return rc, h

    def total_energy_mj(self, handle):
        e = ctypes.c_ulonglong(0)
        rc = self.L.nvmlDeviceGetTotalEnergyConsumption(handle, ctypes.byref(e))
        return rc, int(e.value)


class EnergyMeter:
    """Cumulative device energy in joules; ``available`` is False when NVML or the counter is
    missing (then ``joules()`` returns None and callers report no energy)."""

    def __init__(self, uuid: str, nvml=None):
        self.available = False
        self.reason = ""
        try:
            self.nvml = nvml if nvml is not None else _NvmlLib()
        except OSError as exc:
            self.nvml = None
            self.reason = f"NVML not loadable: {exc}"
            return
        if self.nvml.init() != 0:
            self.reason = "nvmlInit failed"
            return
        rc, self.handle = self.nvml.handle_by_uuid(uuid)
        if rc != 0:
            self.reason = f"no NVML device with UUID {uuid} (status {rc})"
            return
        rc, _ = self.nvml.total_energy_mj(self.handle)
        if rc != 0:
            self.reason = f"total-energy counter not supported (status {rc})"
            return
        self.available = True

    def joules(self):
        if not self.available:
            return None
        rc, mj = self.nvml.total_energy_mj(self.handle)
        return mj / 1e3 if rc == 0 else None

    def close(self):
        if self.nvml is not None:
            self.nvml.shutdown()
            self.nvml = None
            self.available = False


def device_uuid(device) -> str:
    """NVML's UUID string ("GPU-...") of a torch CUDA device."""
    import torch
    u = str(torch.cuda.get_device_properties(device).uuid)
    return u if u.startswith("GPU-") else "GPU-" + u


def measure(meter: EnergyMeter, work, lups_per_call: float, min_seconds: float = 2.0, sync=None,
            clock=time.perf_counter):
    """Run ``work()`` repeatedly for at least ``min_seconds`` (the counter updates in steps of
    tens of milliseconds) and return energy per LUP and mean power over those calls:
    {"pj_per_lup", "watts", "joules", "seconds", "calls", "lups"}; None when no meter."""
    if meter is None or not meter.available:
        return None
    if sync is not None:
        sync()
    e0 = meter.joules()
    t0 = clock()
    calls = 0
    while True:
        work()
        calls += 1
        if sync is not None:
            sync()
        if clock() - t0 >= min_seconds:
            break
    t1 = clock()
    e1 = meter.joules()
    if e0 is None or e1 is None or e1 < e0:
        return None
    joules, secs = e1 - e0, t1 - t0
    lups = lups_per_call * calls
    return {"pj_per_lup": joules / lups * 1e12, "watts": joules / secs, "joules": joules,
            "seconds": secs, "calls": calls, "lups": lups}


def idle_watts(meter: EnergyMeter, seconds: float = 1.0, sleep=time.sleep, clock=time.perf_counter):
    """Mean board power with nothing of ours running (the static share of every figure)."""
    if meter is None or not meter.available:
        return None
    e0, t0 = meter.joules(), clock()
    sleep(seconds)
    e1, t1 = meter.joules(), clock()
    if e0 is None or e1 is None or e1 < e0 or t1 <= t0:
        return None
    return (e1 - e0) / (t1 - t0)
