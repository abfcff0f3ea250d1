"""Seeded synthetic stereo inputs shared by the oracle, the tests and the benchmark."""
from .scenes import (BATCH8, WORKLOADS, batch8_pair, make_pair, random_labels, render_batch8,  # noqa: F401
                     workload_pair)
