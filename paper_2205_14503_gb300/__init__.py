"""GB300-native Voronoi-cell 2-approximation Steiner tree hot path.

The CUDA library is loaded lazily by :mod:`paper_2205_14503_gb300.steiner`
so that the workload generators can be imported on hosts without a GPU.
"""
