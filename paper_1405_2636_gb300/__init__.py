"""GB300-native supernodal sparse direct factorization.

The library ``libspx.so`` (C ABI, declared in ``include/spx.h``) holds the
host analysis and the sm_103a CUDA kernels; ``spx`` is its thin Python
binding.  ``inputs`` draws the seeded synthetic workloads; ``replicas`` holds
the host logic of runs on several GPUs (replicas, shards of a batch).
"""
__all__ = ["spx", "inputs", "replicas"]
