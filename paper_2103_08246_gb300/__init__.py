"""GB300-native fractional-step immersed-boundary Navier--Stokes solver.

The solver lives in a C-ABI shared library built from ``csrc/`` (CUDA for
sm_103a); ``binding`` loads it with ctypes and marshals arguments. Importing
the package does not load the library; ``binding.load()`` does, and fails
loudly if it has not been built.
"""
