"""CPU oracle for the hash containers.  TEST INFRASTRUCTURE ONLY: used by the
tests, the smoke check and the benchmark's CPU-baseline leg; the library never
imports it."""
from .oracle import OracleTable, build, load  # noqa: F401
