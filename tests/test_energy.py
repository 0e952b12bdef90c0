"""Energy-per-LUP bookkeeping (NVML total-energy counter) against a fake NVML on the CPU."""
from paper_1410_5561_gb300 import energy


class FakeNvml:
    """Counter in millijoules that advances by `watts` x simulated seconds."""

    def __init__(self, watts=500.0, uuid="GPU-abc", supported=True, init_rc=0):
        self.watts, self.uuid, self.supported, self.init_rc = watts, uuid, supported, init_rc
        self.t = 0.0
        self.calls = []

    def init(self):
        self.calls.append("init")
        return self.init_rc

    def shutdown(self):
        self.calls.append("shutdown")
        return 0

    def handle_by_uuid(self, uuid):
        return (0, "h") if uuid == self.uuid else (13, None)

    def total_energy_mj(self, handle):
        assert handle == "h"
        if not self.supported:
            return 3, 0
        return 0, int(round(self.watts * self.t * 1e3))

    def clock(self):
        return self.t

    def advance(self, s):
        self.t += s


def test_energy_per_lup_and_power():
    nv = FakeNvml(watts=800.0)
    m = energy.EnergyMeter("GPU-abc", nvml=nv)
    assert m.available
    # each call: 1e9 LUPs in 0.25 s at 800 W -> 200 J -> 200 nJ/LUP = 2e5 pJ/LUP
    r = energy.measure(m, lambda: nv.advance(0.25), 1e9, min_seconds=1.0, clock=nv.clock)
    assert r["calls"] == 4
    assert abs(r["watts"] - 800.0) < 1e-6
    assert abs(r["pj_per_lup"] - 2e5) < 1e-3
    assert abs(r["joules"] - 800.0) < 1e-6
    w = energy.idle_watts(m, seconds=2.0, sleep=nv.advance, clock=nv.clock)
    assert abs(w - 800.0) < 1e-6
    m.close()
    assert nv.calls[-1] == "shutdown" and not m.available
    assert m.joules() is None


def test_unavailable_meter_reports_nothing():
    for nv, why in [(FakeNvml(uuid="GPU-other"), "no NVML device"),
                    (FakeNvml(supported=False), "not supported"),
                    (FakeNvml(init_rc=1), "nvmlInit failed")]:
        m = energy.EnergyMeter("GPU-abc", nvml=nv)
        assert not m.available and why in m.reason
        assert m.joules() is None
        assert energy.measure(m, lambda: None, 1.0) is None
        assert energy.idle_watts(m) is None
    assert energy.measure(None, lambda: None, 1.0) is None


def test_counter_reset_is_not_reported_as_energy():
    nv = FakeNvml(watts=100.0)
    m = energy.EnergyMeter("GPU-abc", nvml=nv)

    def work():  # the counter goes backwards (driver reload)
        nv.watts = -100.0
        nv.advance(1.0)

    assert energy.measure(m, work, 1.0, min_seconds=0.5, clock=nv.clock) is None
