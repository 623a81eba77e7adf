"""GB300-native spectral/hp element operators (mass, Laplacian, Helmholtz on
mixed hex/prism/pyramid/tet meshes) behind a C ABI (libhp.so).

Submodules:
  inputs  seeded synthetic meshes and coefficients (no operator arithmetic)
  hp      ctypes binding of the C ABI declared in include/hp.h
  build   compiles libhp.so for sm_103a in-tree
Importing the package loads nothing; ``paper_2604_04644_gb300.hp`` loads the library.
"""
