"""The generator voltage V(t) = V0 sin(2 pi f t) of the lumped gap feed at
step k (t = k dt), as the tests need it to set up electrostatic boundary
values on the host; the library evaluates the same waveform itself."""
import math


def drive_voltage(cfg, step):
    t = step * cfg["dt"]
    return cfg["volt"] * math.sin(2.0 * math.pi * cfg["freq"] * t)
