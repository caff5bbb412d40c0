"""GB300-native hash-partitioned shuffle + inner hash join (the data-parallel
hot path of the cuDF merge workload in arXiv 2101.08878, Sec. V-B).

The compute path is ``libmdj.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/mdj.h``); ``paper_2101_08878_gb300.mdj`` is its thin
ctypes binding.  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["mdj", "datagen"]
