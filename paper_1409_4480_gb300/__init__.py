"""GB300-native Lyman-alpha Monte-Carlo radiative transfer (the COLT packet
loop of Smith et al. 2014) behind a C-ABI CUDA library.

`colt` holds the binding to libcolt.so; `synth` the seeded input generators.
"""
