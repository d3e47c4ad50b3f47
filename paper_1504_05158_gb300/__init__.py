"""GB300-native multi-swarm PSO for the Quadratic Assignment Problem.

The compute path lives in the CUDA library ``libqap_pso.so`` (sources in
``csrc/``); :mod:`paper_1504_05158_gb300.qap_pso` is its thin ctypes binding.
Importing the package does not load the library; the binding loads it on first
use and raises if it is missing.
"""
