"""Seeded synthetic stereo inputs shared by the oracle, the tests and the benchmark."""
from .scenes import make_pair, workload_pair, random_labels, WORKLOADS  # noqa: F401
