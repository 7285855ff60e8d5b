"""B300 (sm_103a) hot path of the paper's data-mapping analysis.

Thin Python binding over ``libodp.so`` (C ABI declared in ``include/odp.h``):
argument marshalling only -- every step runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  The compiled library is loaded
on first use of any binding name and its absence raises ImportError; there
is no CPU fallback.  ``paper_2601_12713_b300.build`` compiles it.
"""

_EXPORTS = (
    "LIB_PATH", "lib", "status_string", "OdpError", "fingerprint", "fingerprint_one",
    "fingerprint_noalloc", "fingerprint_log", "fingerprint_tensors", "fingerprint_with", "autotune_fingerprint", "autotune_clear",
    "fingerprint_status", "analyze", "Findings", "EVENT_DTYPE", "FINDING_DTYPE", "SITE_DTYPE",
    "SUMMARY_FIELDS", "set_torch_allocator", "release_scratch", "Server", "log_tensor",
    "verify_fingerprints", "set_allocator", "server_bytes",
)


def __getattr__(name):
    if name in _EXPORTS:
        from . import _lib

        return getattr(_lib, name)
    raise AttributeError(name)


def __dir__():
    return sorted(list(_EXPORTS) + ["build"])
