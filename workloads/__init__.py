"""Seeded synthetic input generators shared by the tests, the oracle and the
benchmark.  Nothing here implements hash-container behaviour."""
from . import splitmix, recipes  # noqa: F401
