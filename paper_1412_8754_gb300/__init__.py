"""GB300-native free-energy engine for the two-band FFLO model (arXiv:1412.8754).

The compute path is the C-ABI library libffe.so (include/ffe.h) built from
csrc/*.cu for sm_103a; ``ffe`` is its ctypes binding and ``workloads`` holds
the seeded synthetic inputs.  Importing the package does not load the
library; the first call into ``ffe`` does, and fails loudly if it is absent.
"""
from . import workloads  # noqa: F401

__all__ = ["ffe", "workloads", "build"]
