"""GB300-native differentiable IDM traffic simulator (arXiv 2412.16750).

The compute path is the C-ABI library ``libidm`` built from ``csrc/`` for
sm_103a; ``paper_2412_16750_gb300.lib`` binds it and fails loudly when it is
missing.  Importing this package loads nothing; ``synth`` (seeded inputs)
needs no GPU.
"""
