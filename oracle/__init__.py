"""Oracle for the MBE-FCI tuple-CASCI hot path.

TEST INFRASTRUCTURE ONLY.  A plain, slow, CPU implementation of what the CUDA
path computes, written from the method's definitions:

* ``fci``  -- determinant-basis CASCI from the Slater-Condon rules (C core in
  fci.c, built by build.py with gcc) with a library eigensolver;
* ``mbe``  -- reference energy, frozen-core active-space Hamiltonian, tuple
  enumeration and skip rule, tuple energies, the increment recursion (Eq. 2)
  and the order sums and totals (Eqs. 1 and 3).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference leg of ``bench.py`` may import anything here.  The product package
never does, and shares no code with this directory.

Parity pins (tests/test_oracle_*.py) tie these functions to facts outside the
oracle itself: closed forms of the Hubbard model, a brute-force Fock-space
Hamiltonian built from fermion operator matrices, frozen-core FCI in the full
orbital space, the Moebius-inversion identity of Eqs. 1-2 at full order, and
combinatorial counts.  Functions without such a pin are marked "parity
unpinned" in their docstrings.
"""
