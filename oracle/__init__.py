"""CPU oracle for the DSRG-MRPT2/PT3 energy (plain, slow, FP64).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with
the CUDA library.

Modules
-------
mkgno     generic Mukherjee-Kutzelnigg normal-ordered commutator engine on
          dense spin-orbital tensors (Sec. II, Eq. exactBCH and the 1,2-body
          truncation; the paper defers the term list, so the engine
          enumerates the generalized Wick contractions itself).
fockspace brute-force Fock-space operators used to pin the engine.
dsrg      the DSRG-MRPT2/PT3 energy (Sec. II.B, Eqs. Hbar_0th..E(3),
          T1_1st..T2_2nd) on top of the engine.
"""
