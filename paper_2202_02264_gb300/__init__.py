"""dSMC (de-Sequentialized Monte Carlo, arXiv 2202.02264) for GB300 (sm_103a).

The hot path lives in the CUDA library ``libdsmc.so`` (C ABI: include/dsmc.h); ``dsmc``
is its thin binding and ``workloads`` the seeded synthetic inputs.
"""
