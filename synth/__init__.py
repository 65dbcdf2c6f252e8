"""Seeded synthetic inputs (noise + pulse trains) and named workloads.

Shared by tests and benchmark; contains no dedispersion arithmetic."""
from .voltages import PulseTrain, complex_int8_voltages  # noqa: F401
from .workloads import WORKLOADS, Workload  # noqa: F401
