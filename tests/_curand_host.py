"""Calls NVIDIA cuRAND's host-side (CPU) Philox4x32-10 generator through ctypes.

cuRAND is an independent implementation of Philox4x32-10; its host generator
runs on the CPU, so it pins the oracle's Philox without a GPU.  Nothing is
copied from it: it is only called.
"""
import ctypes
import glob
import os

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _find():
    cands = []
    for root in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if root:
            cands += sorted(glob.glob(os.path.join(root, "lib64", "libcurand.so*")))
            cands += sorted(glob.glob(os.path.join(root, "targets", "*", "lib", "libcurand.so*")))
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def philox_host_words(seed: int, nwords: int, offset: int = 0):
    """First nwords 32-bit outputs of cuRAND's host Philox generator, or None."""
    L = _find()
    if L is None:
        return None
    gen = ctypes.c_void_p()
    if L.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        return None
    try:
        if L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) != 0:
            return None
        if offset and L.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) != 0:
            return None
        buf = (ctypes.c_uint32 * nwords)()
        if L.curandGenerate(gen, buf, ctypes.c_size_t(nwords)) != 0:
            return None
        return list(buf)
    finally:
        L.curandDestroyGenerator(gen)
