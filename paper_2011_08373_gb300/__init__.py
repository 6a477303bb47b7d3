"""GB300-native engine for the barrier-repair loop of GPURepair (Joshi and
Muduganti, arXiv 2011.08373): an exact all-threads race/divergence check, a
clause builder and an exact minimum-weight hitting-set search, driven to a
fixed point on the device (Algorithm 1), behind the C ABI in
``include/gpurepair.h``.

Importing the package loads nothing native; ``paper_2011_08373_gb300.binding``
loads ``libgpurepair.so`` on first use and raises if it is missing.
"""

__all__ = ["synth", "binding"]
