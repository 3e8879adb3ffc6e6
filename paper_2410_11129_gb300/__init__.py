"""GB300-native coupled time step of the ferrofluid compound droplet model
(arXiv 2410.11129): phase-field MRT lattice Boltzmann + magnetic potential.

The CUDA library (libfcd.so, C-ABI in include/fcd.h) is loaded lazily by
``paper_2410_11129_gb300.fcd``; ``workloads`` holds the synthetic inputs.
"""
