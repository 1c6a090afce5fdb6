"""GB300-native MG-sketch local-moving sweep (Louvain / Leiden / LPA).

The compute path is the CUDA library behind ``include/cd.h``; the Python
binding in :mod:`paper_2411_02268_gb300.cd` only marshals arguments.
"""
