"""Seeded synthetic inputs shared by the oracle tests, the parity tests and the
benchmark.  Draws and layouts only; no transport arithmetic lives here."""
from .junction import (ANGSTROM, RYDBERG_EV, Instance, Lead, minimal_cell, junction,
                       junction_ecut_for, explicit_barrier, explicit_tables, random_tables,
                       random_points, uneven_batch)

__all__ = ["ANGSTROM", "RYDBERG_EV", "Instance", "Lead", "minimal_cell", "junction",
           "junction_ecut_for", "explicit_barrier", "explicit_tables", "random_tables",
           "random_points", "uneven_batch"]
