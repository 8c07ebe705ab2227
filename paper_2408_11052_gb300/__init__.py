"""GB300-native contrastive-RL (CRL) update step (arXiv 2408.11052).

The compute lives in ``libcrl.so`` (CUDA kernels for sm_103a behind the C ABI
of ``include/crl.h``); this package only marshals arguments.  Importing the
package does not load the library; ``paper_2408_11052_gb300.api`` does, and
fails loudly when it is missing.
"""

__all__ = ["api", "functional", "workload", "build"]
