"""Independent XXH64 for pinning the oracle: the system's libxxhash, if present."""
import ctypes
import ctypes.util

_lib = None


def load():
    """Return a callable xxh64(bytes, seed) from libxxhash, or None if absent."""
    global _lib
    if _lib is None:
        names = [ctypes.util.find_library("xxhash"), "libxxhash.so.0", "libxxhash.so"]
        for nm in names:
            if not nm:
                continue
            try:
                L = ctypes.CDLL(nm)
                L.XXH64.restype = ctypes.c_uint64
                L.XXH64.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
                _lib = L
                break
            except OSError:
                continue
    if _lib is None:
        return None

    def h(data, seed=0):
        b = bytes(data)
        return int(_lib.XXH64(b, len(b), seed))
    return h
