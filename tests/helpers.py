"""Test-only re-exports shared by the GPU parity tests."""
from workloads import random_canonical_mps  # noqa: F401
