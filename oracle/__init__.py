"""Plain, slow FP64 CPU oracle for the M-scheme block Hamiltonian product and
the thick-restart block Lanczos eigensolver (Shimizu et al., arXiv 1902.02064).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this package: only the tests, the smoke check and the benchmark's CPU baseline
do.  It shares no code with the CUDA library; the only module both sides use is
``synth`` (seeded inputs, no arithmetic of the method).

Contents
--------
basis        determinant enumeration (Sec. II Eq. (mbasis); App. A Table I,
             Eq. (part)) and a generating-function dimension count.
hamiltonian  explicit H assembly by applying every operator term of the
             Hamiltonian (Sec. II, App. B.1 Eq. (twobodybit), App. B.2
             Eq. (pntwobodybit)) to every determinant, with fermion signs
             from the Jordan-Wigner ordering; sampled rows of H.V.
jw           an independent Jordan-Wigner matrix construction of the same H
             (used only to pin the bit-string assembly on tiny spaces).
lanczos      Algorithm 1 (Lanczos) with full reorthogonalisation, dense eigh,
             spectral norm.
gradient     Hellmann-Feynman expectation <v|dH/dtheta|v> per parameter.
"""
