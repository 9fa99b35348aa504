"""GB300-native matrix probing: H = F*F on batches of trial functions, the
randomized fit of a pseudodifferential approximation of H^{-1}, and its
application as a preconditioner (Demanet et al., matrix probing).

The compute path is the sm_103a CUDA library ``_lib/libprobe.so`` behind the C
ABI of ``include/probe.h``; :mod:`.binding` is its thin ctypes binding and
:mod:`.autograd` exposes the nonlinear forward map as a differentiable torch
function whose backward is the adjoint kernel.  Importing this package fails
if the library has not been built.
"""
from .binding import (  # noqa: F401
    Basis,
    Probe,
    ProbeError,
    apply_H_group,
    lib,
    probe_version,
)

from .autograd import ForwardMap, forward_map, misfit  # noqa: F401,E402

__all__ = ["Basis", "Probe", "ProbeError", "apply_H_group", "lib", "probe_version", "ForwardMap",
           "forward_map", "misfit"]
