"""Zero-copy export of library-owned device buffers through DLPack (§3.3).

A DLManagedTensor (pointer, shape, dtype, device) is built in host memory and
wrapped in a "dltensor" capsule; torch.from_dlpack then views the same device
memory without copying. The buffer stays owned by the library: the view must
not outlive the result it came from (sift_serve_release frees it).
"""
from __future__ import annotations

import ctypes
from ctypes import CFUNCTYPE, POINTER, Structure, c_int, c_int64, c_uint8, c_uint16, c_uint64, c_void_p

_KDL_CUDA = 2
_DTYPES = {"f32": (2, 32), "i32": (0, 32)}


class _DLDevice(Structure):
    _fields_ = [("device_type", c_int), ("device_id", c_int)]


class _DLDataType(Structure):
    _fields_ = [("code", c_uint8), ("bits", c_uint8), ("lanes", c_uint16)]


class _DLTensor(Structure):
    _fields_ = [("data", c_void_p), ("device", _DLDevice), ("ndim", c_int), ("dtype", _DLDataType),
                ("shape", POINTER(c_int64)), ("strides", POINTER(c_int64)),
                ("byte_offset", c_uint64)]


_Deleter = CFUNCTYPE(None, c_void_p)


class _DLManagedTensor(Structure):
    _fields_ = [("dl_tensor", _DLTensor), ("manager_ctx", c_void_p), ("deleter", _Deleter)]


_alive = {}


@_Deleter
def _deleter(ptr):
    _alive.pop(ptr, None)


_PyCapsule_New = ctypes.pythonapi.PyCapsule_New
_PyCapsule_New.restype = ctypes.py_object
_PyCapsule_New.argtypes = [c_void_p, ctypes.c_char_p, c_void_p]


def capsule(ptr: int, shape, dtype: str, device_id: int):
    """A DLPack capsule viewing `ptr` (device memory) as a C-contiguous tensor."""
    code, bits = _DTYPES[dtype]
    nd = len(shape)
    shp = (c_int64 * nd)(*shape)
    mt = _DLManagedTensor()
    mt.dl_tensor.data = ptr
    mt.dl_tensor.device = _DLDevice(_KDL_CUDA, device_id)
    mt.dl_tensor.ndim = nd
    mt.dl_tensor.dtype = _DLDataType(code, bits, 1)
    mt.dl_tensor.shape = shp
    mt.dl_tensor.strides = None
    mt.dl_tensor.byte_offset = 0
    mt.deleter = _deleter
    addr = ctypes.addressof(mt)
    _alive[addr] = (mt, shp)
    return _PyCapsule_New(addr, b"dltensor", None)


def device_tensor(ptr, shape, dtype: str, device_id: int):
    import torch  # noqa: PLC0415
    n = 1
    for s in shape:
        n *= s
    if n == 0 or not ptr:
        tdt = torch.float32 if dtype == "f32" else torch.int32
        return torch.empty(shape, dtype=tdt, device=torch.device("cuda", device_id))
    return torch.utils.dlpack.from_dlpack(capsule(ptr, shape, dtype, device_id))
