"""GB300-native dictionary learning with Jacobi atom updates (arXiv 1509.05054).

The compute path is the C-ABI library built from ``csrc/`` (hand-written
sm_103a CUDA kernels); :mod:`paper_1509_05054_gb300.dl` is its thin Python
binding.  :mod:`paper_1509_05054_gb300.synth` draws the seeded inputs.
"""
__all__ = ["synth"]
