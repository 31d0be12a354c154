"""GB300-native semi-implicit Fourier-spectral phase-field step (CUDA, sm_103a).

Import `paper_2306_04322_gb300.fs` for the C-ABI binding; `inputs` holds the
seeded synthetic workloads.  Importing the package itself loads no native code.
"""
