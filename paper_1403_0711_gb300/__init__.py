"""GB300-native lattice path-integral Coulomb energy sampler.

Sugihara, Higo & Nakamura, "Local Representation of N-body Coulomb Energy
with Path Integrals" (JPSJ 2014): the N-body Coulomb energy as the free-field
expectation value Eq. (nsum), sampled by heatbath / over-relaxation Markov
chains on a Dirichlet cubic lattice.

  coulps   binding of the C ABI in include/coulps.h (libcoulps.so)
  inputs   seeded synthetic charge sets
"""
__all__ = ["coulps", "inputs"]
