"""Exact betweenness centrality on one GB300 (sm_103a).

The compute path is the shared library built from ``csrc/`` (C-ABI declared in
``include/bc_gb300.h``); :mod:`paper_0809_1906_gb300.native` marshals arguments
to it. :mod:`paper_0809_1906_gb300.graphs` generates seeded inputs.
"""
