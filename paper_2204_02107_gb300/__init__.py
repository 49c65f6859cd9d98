"""GB300-native incompressible-flow time step of DNSLABIB (arXiv 2204.02107) for indoor-ventilation rooms.

The step runs in hand-written CUDA kernels for sm_103a behind the C ABI in ``include/ventflow.h``;
``native`` is its ctypes binding (argument marshalling only), ``rooms`` builds seeded synthetic inputs, and
``serve`` runs many rooms as a continuous-batching request loop.
"""
__all__ = ["native", "rooms"]
