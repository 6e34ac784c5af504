"""GB300-native forward/adjoint/gradient solver for the tumor
reaction-diffusion model of image-driven tumor-growth calibration.

The compute path is the C-ABI library ``librd`` (CUDA, sm_103a) built from
``csrc/``; :mod:`.rd` is its thin ctypes binding and :mod:`.synth` holds the
seeded synthetic input recipes.  Importing the package does not load the
library; :func:`paper_1907_07774_gb300.rd.lib` does, and fails loudly when it
is missing.
"""
