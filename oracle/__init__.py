"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle of the CI-SCvx discretization.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
and reference legs) may import this package.  The product package never
imports it, and it imports nothing from the product package: robots come in as
plain dictionaries of numpy arrays (the shared seeded generator builds them).

The arithmetic lives in ``oracle.cpp`` (compiled with g++); this module only
marshals arrays.  See the header of ``oracle.cpp`` for what is computed and the
paper passages each step follows.
"""
from .oracle import (  # noqa: F401
    OracleModel,
    build,
    dims,
    discretize,
    flow,
    interval,
    linear_interval,
    node,
    node_value,
    psi,
    rhs,
    tableau,
    vjp,
)
