"""FP64 reference ("oracle") for the split-explicit barotropic subcycle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``. The library under ``paper_2311_08241_gb300`` never
imports, links or runs anything in this directory, and shares no code with it.

Contents:
    oracle.c   plain C, FP64, edge-form (median-dual) substeps of Eq. (4.10), the
               time mean of Eq. (4.12), volume/energy diagnostics.
    runner.py  build (gcc) and ctypes wrapper of oracle.c.
    brute.py   numpy dense-matrix brute force for tiny meshes (finite-element
               gradient and its adjoint, one linear solve per substep).
    closed.py  closed forms of the paper's Sect. 3 (characteristic matrix of the
               SE scheme, its polynomial, small-Courant expansion).

Parity status: every function here is pinned by the tests in ``tests/test_oracle_*.py``
against closed forms, invariants and brute force; none is "parity unpinned".
"""
