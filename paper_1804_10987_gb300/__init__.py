"""GB300-native feedforward decentralized precoding (arXiv:1804.10987).

The compute path lives in the CUDA library ``libdprecode.so`` behind the C ABI
declared in ``include/dprecode.h``; ``paper_1804_10987_gb300.dp`` is the thin
Python binding over it.  ``synth`` draws the seeded synthetic inputs.
"""
__all__ = ["dp", "synth"]
