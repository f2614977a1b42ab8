"""GB300-native deterministic multilevel process mapping (integrated mapping,
Section 4.2 of "GPU-Accelerated Algorithms for Process Mapping").

``gpumap`` binds the CUDA library (C ABI in ``include/gpumap.h``);
``inputs`` builds the seeded synthetic workloads.  Importing the package does
not load the library; the first ``gpumap`` call does (and raises if it cannot).
"""
