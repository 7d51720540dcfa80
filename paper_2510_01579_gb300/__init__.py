"""GB300 (sm_103a) implementation of the MMGaP hot path: delta-Ising build,
CIM-CAC anneals and decode for uplink MIMO detection and downlink
vector-perturbation precoding, behind the C ABI of include/mmgap.h.

``Context``, ``Params`` and ``MMGaPError`` come from the ctypes binding, which
is imported on first use and raises if the CUDA library has not been built.
"""
__all__ = ["Context", "Params", "MMGaPError", "SUPPORTED_NT", "Batch", "Server", "VARIANT_NAMES"]


def __getattr__(name):
    if name in __all__:
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
