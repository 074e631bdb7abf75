"""GB300-native sector-signature data carving (hash every 512-byte disk sector, look the digest
up in a table built from known master files, report every match).

The compute path is the C-ABI library ``libcv.so`` built from ``csrc/`` (hand-written sm_103a
CUDA); :mod:`paper_0901_1307_gb300.cv` is its thin Python binding. ``synth`` generates seeded
synthetic inputs.
"""
