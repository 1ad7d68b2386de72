"""GB300-native domain-decomposed stochastic estimate of fermion determinant ratios.

Finkenrath, Knechtli, Leder, "Application of Domain Decomposition to the Evaluation of Fermion
Determinant Ratios" (Lattice 2012): the two-flavour mass-reweighting factor 1/det(Mh^dag Mh)
through the black/white block Schur complement of the Wilson-clover operator.

* ``binding`` -- the Python binding of the C ABI (``include/ddrw.h``) of the CUDA library;
* ``build``   -- compiles ``csrc/*.cu`` for sm_103a into ``_build/libddrw.so``;
* ``synth``   -- seeded synthetic inputs (gauge fields, spinors).
"""
__all__ = ["binding", "build", "synth"]
