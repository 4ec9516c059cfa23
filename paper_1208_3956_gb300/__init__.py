"""GB300-native double-sweep PML domain-decomposition Helmholtz solver.

The solver is the C-ABI library libhelmdd.so (include/helm_dd.h); ``helm`` is
its Python binding and ``media`` the seeded synthetic inputs.  Importing the
package does not load the library; ``paper_1208_3956_gb300.helm.load()`` does,
and raises when it has not been built.
"""
