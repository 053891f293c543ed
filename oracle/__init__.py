"""CPU FP64 oracle for the overlap operator -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct numpy restatement of what the library
computes, written from the paper (Lujan, Alexandru, Lee, "Electric
polarizability of hadrons with overlap fermions on multi-GPUs", Lattice 2011)
and from textbook lattice QCD where the paper is silent.  Every function cites
the passage it follows.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  The library (``paper_1111_6288_gb300``)
never imports it and shares no code with it; both only read the seeded inputs
from ``synth``.

Modules
-------
``dirac``      gamma matrices, Wilson D_w and H_w = gamma5 D_w (Sec. 2, eq. 1)
``chebyshev``  the polynomial P(x) ~ x^{-1/2} and the error law (Sec. 2, eq. 2)
``overlap``    sign(H_w) with the small/large space split, D_ov, D(m) (Sec. 2)
``solver``     CG on the normal equations for D(m) x = b (Sec. 3.2)
``dense``      dense-matrix tools for tiny lattices (exact references)
``correlator`` pion correlator from point-source propagators (Sec. 4)

Every function here is pinned by a ``-m "not gpu"`` test against a closed
form, an invariant, a library routine or a value the paper prints.
"""
