"""Seeded, synthetic problem definitions shared by the CUDA path's tests and the oracle.

This package only *describes* problems: which modes, which normal-ordered Hamiltonian
monomials, which jump operators, which measured operator, which drive envelopes and
which seeds.  It performs none of the method's arithmetic (no mapping, no generator,
no time stepping, no envelope evaluation), so both sides can consume it without
sharing any of the computation they are compared on.
"""

from .spec import Channel, HTerm, Jump, Problem  # noqa: F401
from . import configs  # noqa: F401
