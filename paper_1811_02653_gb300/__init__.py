"""GB300-native OverSketch: C ~= (A S)(S^T B) with straggler masks.

The compute path is the C-ABI library ``liboversketch.so`` built from
``csrc/`` (hand-written sm_103a CUDA).  This package is the thin binding:
argument marshalling only, no arithmetic of the method.  Importing the
package does not load the library; the first call through ``ops`` does, and
fails loudly when it is missing.
"""
__all__ = ["ops", "workloads"]
