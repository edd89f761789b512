"""CPU oracle for the random-circuit amplitude path.

This package is test infrastructure.  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the library itself never
does, and it shares no code with the CUDA path.

Everything is plain NumPy in float64 / complex128, written for a reader to
check against the paper and against textbook quantum mechanics:

* ``gates``       -- gate matrices of the benchmark gate set.
* ``circuit``     -- the seeded random-circuit protocol (own SplitMix64).
* ``statevector`` -- state-vector simulation: amplitude <x|U|0...0>.
* ``tn``          -- an independent tensor-network contractor with its own
                     network builder, its own greedy order and exact slicing
                     (Sec. "A PEPS-based Simulation Method with an Optimized
                     Slicing Strategy": the sum over all 2^S assignments of the
                     sliced indices equals the unsliced contraction).
* ``stats``       -- Porter-Thomas moments and linear XEB (Sec. "Result
                     Validation with Different Precisions"; Appendix A).

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute force, identities); see the test files named
``test_oracle_*``.
"""
