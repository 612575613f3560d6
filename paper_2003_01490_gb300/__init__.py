"""GB300-native four-way coupled lattice Boltzmann / discrete element method.

The compute path is the CUDA library built from ``csrc/`` (see
``build.py``) behind the C ABI of ``include/lbmdem.h``; ``lbmdem`` is its
Python binding and ``workloads`` the seeded synthetic input generators.
``serve`` runs a stream of independent jobs with continuous batching, and
``validation`` runs the full-size cases that compare with the paper's
printed results. Importing the package loads nothing;
``lbmdem.load_library()`` loads the shared library on first use.
"""
