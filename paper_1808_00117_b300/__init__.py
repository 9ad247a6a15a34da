"""Python binding of the B300 capture/restore library (libcrum.so).

Argument marshalling only: every step of the path runs in the CUDA library
behind ``include/crum.h``.  Functions keep the C names (``crum_register``,
``crum_checkpoint`` ...); ``CheckpointSet`` and ``Image`` wrap the handles.
Pointers are plain integers (``tensor.data_ptr()``, ``stream.cuda_stream``).

Importing never builds; ``load()`` raises ``ImportError`` when the compiled
library is absent, so a missing extension fails loudly instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

__all__ = [
    "load", "CrumError", "CheckpointSet", "Image", "Config", "ImageInfo",
    "FULL", "INCR", "VERIFY", "WAIT_CAPTURED", "WAIT_DRAINED", "WAIT_PERSISTED",
    "SINK_MEMORY", "SINK_FILE", "SINK_NULL", "PAGE_SIZE", "NO_PARENT",
]

PAGE_SIZE = 65536
NO_PARENT = 0xFFFFFFFFFFFFFFFF
INCR, FULL, VERIFY, NO_PAYLOAD = 0, 1, 2, 4
WAIT_CAPTURED, WAIT_DRAINED, WAIT_PERSISTED = 1, 2, 3
SINK_MEMORY, SINK_FILE, SINK_NULL = 0, 1, 2
RESTORE_AUTO, RESTORE_REPLAY, RESTORE_MERGED, RESTORE_DELTA = 0, 1, 2, 3
NUM_HASH_MAPPINGS, NUM_GATHER_MAPPINGS = 15, 6  # CRUM_NUM_HASH_MAPPINGS, CRUM_NUM_GATHER_MAPPINGS

STATUS = {0: "CRUM_OK", 1: "CRUM_EINVAL", 2: "CRUM_ENOMEM", 3: "CRUM_EBUSY", 4: "CRUM_ECUDA",
          5: "CRUM_EIO", 6: "CRUM_EMISMATCH", 7: "CRUM_ECOLLISION", 8: "CRUM_ETIMEOUT",
          9: "CRUM_ECORRUPT"}
OK, EINVAL, ENOMEM, EBUSY, ECUDA, EIO, EMISMATCH, ECOLLISION, ETIMEOUT, ECORRUPT = range(10)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcrum.so")


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("staging_bytes", ctypes.c_uint64),
                ("chunk_bytes", ctypes.c_uint64), ("host_pool_bytes", ctypes.c_uint64),
                ("sink", ctypes.c_int), ("sink_dir", ctypes.c_char_p),
                ("verify", ctypes.c_int), ("fsync", ctypes.c_int),
                ("hash_mapping", ctypes.c_int), ("gather_mapping", ctypes.c_int),
                ("external_staging", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("max_chain", ctypes.c_int), ("restore_mode", ctypes.c_int),
                ("max_pending", ctypes.c_int), ("compress", ctypes.c_int),
                ("managed_in_place", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("staging_budget", ctypes.c_uint64),
                ("max_inflight", ctypes.c_int), ("max_checkpoints", ctypes.c_int),
                ("max_restores", ctypes.c_int), ("serialize_drains", ctypes.c_int),
                ("order", ctypes.c_int), ("keep_images", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("client", ctypes.c_uint32), ("kind", ctypes.c_int),
                ("status", ctypes.c_int), ("done", ctypes.c_int), ("n_dirty", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64), ("image_seq", ctypes.c_uint64),
                ("checksum", ctypes.c_uint64),
                ("t_queue_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("bytes_checkpointed", ctypes.c_uint64),
                ("bytes_restored", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("p50_ckpt_ms", ctypes.c_double),
                ("p99_ckpt_ms", ctypes.c_double), ("p50_restore_ms", ctypes.c_double),
                ("p99_restore_ms", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("peak_inflight", ctypes.c_uint32), ("peak_staging", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_CHECKPOINT, REQ_CHECKPOINT_FULL, REQ_RESTORE = 0, 1, 2


class ImageInfo(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_uint64), ("parent_seq", ctypes.c_uint64),
                ("n_dirty", ctypes.c_uint64), ("n_pages", ctypes.c_uint64),
                ("image_bytes", ctypes.c_uint64), ("checksum", ctypes.c_uint64),
                ("collisions", ctypes.c_uint64), ("n_allocs", ctypes.c_uint32),
                ("full", ctypes.c_uint32), ("stage", ctypes.c_int), ("status", ctypes.c_int),
                ("t_captured_ms", ctypes.c_double), ("t_drained_ms", ctypes.c_double),
                ("t_persisted_ms", ctypes.c_double), ("t_hash_ms", ctypes.c_double),
                ("t_compact_ms", ctypes.c_double), ("t_drain_ms", ctypes.c_double),
                ("host_pages", ctypes.c_uint64), ("t_encode_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every exported symbol of include/crum.h with its ctypes signature.
_VP, _U64, _U32, _I, _I64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "crum_config_default": ([ctypes.POINTER(Config)], None),
    "crum_last_error": ([], ctypes.c_char_p),
    "crum_version": ([], ctypes.c_char_p),
    "crum_set_create": ([ctypes.POINTER(Config), ctypes.POINTER(_VP)], _I),
    "crum_set_destroy": ([_VP], _I),
    "crum_register": ([_VP, _VP, ctypes.c_size_t, ctypes.POINTER(_U32)], _I),
    "crum_unregister": ([_VP, _U32], _I),
    "crum_set_info": ([_VP, ctypes.POINTER(_U32), ctypes.POINTER(_U64)], _I),
    "crum_autotune": ([_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_double)], _I),
    "crum_checkpoint": ([_VP, _VP, _I, ctypes.POINTER(_VP)], _I),
    "crum_image_wait": ([_VP, _I, _I64], _I),
    "crum_image_info_get": ([_VP, ctypes.POINTER(ImageInfo)], _I),
    "crum_image_copy": ([_VP, _VP, _U64], _I),
    "crum_image_save": ([_VP, ctypes.c_char_p], _I),
    "crum_image_load": ([_VP, ctypes.c_char_p, _VP, ctypes.POINTER(_VP)], _I),
    "crum_image_from_bytes": ([_VP, _VP, _U64, _VP, ctypes.POINTER(_VP)], _I),
    "crum_image_release": ([_VP], _I),
    "crum_restore": ([_VP, _VP, _VP], _I),
    "crum_restore_pages": ([_VP, ctypes.POINTER(_U64)], _I),
    "crum_hash_pages": ([_VP, _U64, _VP, _VP], _I),
    "crum_hash_bytes": ([_VP, _U64, _U64, _VP, _VP], _I),
    "crum_get_hashes": ([_VP, _VP, _U64], _I),
    "crum_poke_hash": ([_VP, _U64, _U64], _I),
    "crum_kernel_launches": ([], _U64),
    "crum_selftest_wait_timeout": ([_VP, _U64, _U64, ctypes.POINTER(_I), _VP], _I),
    "crum_dirty_pages_static": ([_VP, _U64, _VP, _I, _VP, _VP, _VP], _I),
    "crum_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(_VP)], _I),
    "crum_server_destroy": ([_VP], _I),
    "crum_server_add_client": ([_VP, _VP, _VP, ctypes.POINTER(_U32)], _I),
    "crum_server_submit": ([_VP, _U32, _I, ctypes.POINTER(_U64)], _I),
    "crum_server_wait": ([_VP, _U64, _I, _I64, ctypes.POINTER(RequestInfo)], _I),
    "crum_server_take_image": ([_VP, _U64, ctypes.POINTER(_VP)], _I),
    "crum_server_drain": ([_VP, ctypes.POINTER(ServerStats)], _I),
    "crum_server_reset_stats": ([_VP], _I),
}

_lib = None


def load():
    """Load libcrum.so (built by ``paper_1808_00117_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run python -m paper_1808_00117_b300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes, fn.restype = args, res
        _lib = lib
    return _lib


class CrumError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().crum_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


def _check(st: int, where: str, ok=(OK,)):
    if st not in ok:
        raise CrumError(st, where)
    return st


def config(**kw) -> Config:
    c = Config()
    load().crum_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k == "sink_dir" and isinstance(v, str):
            v = v.encode()
        setattr(c, k, v)
    return c


def version() -> str:
    return load().crum_version().decode()


def kernel_launches() -> int:
    return int(load().crum_kernel_launches())


def hash_pages(ptr: int, nbytes: int, out_ptr: int, stream: int = 0) -> None:
    """Page hashes of one device allocation into a device u64 array."""
    _check(load().crum_hash_pages(ptr, nbytes, out_ptr, stream), "crum_hash_pages")


def hash_bytes(ptr: int, nbytes: int, first_index: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().crum_hash_bytes(ptr, nbytes, first_index, out_ptr, stream), "crum_hash_bytes")


def dirty_pages_static(ptr: int, nbytes: int, hashes_ptr: int, full: bool, pages_out_ptr: int,
                       count_out_ptr: int, stream: int = 0) -> None:
    """Changed pages of one allocation with no memory allocated by the
    library (its scratch is a fixed device array; see include/crum.h)."""
    _check(load().crum_dirty_pages_static(ptr, nbytes, hashes_ptr, int(bool(full)), pages_out_ptr,
                                          count_out_ptr, stream), "crum_dirty_pages_static")


def selftest_wait_timeout(ptr: int, nbytes: int, limit_ns: int, stream: int = 0) -> bool:
    """Run the bounded-wait self-test (one bulk copy is never issued);
    True if the kernel reported that its wait ran out and finished."""
    flag = ctypes.c_int(-1)
    _check(load().crum_selftest_wait_timeout(ptr, nbytes, limit_ns, ctypes.byref(flag), stream),
           "crum_selftest_wait_timeout")
    return flag.value == 1


class Image:
    """A checkpoint image handle (library-owned, reference counted)."""

    def __init__(self, handle: int):
        self.handle = handle

    def wait(self, what: int = WAIT_PERSISTED, timeout_s: Optional[float] = None,
             allow=(OK, ECOLLISION)) -> int:
        t = -1 if timeout_s is None else int(timeout_s * 1e9)
        return _check(load().crum_image_wait(self.handle, what, t), "crum_image_wait", allow)

    def info(self) -> dict:
        i = ImageInfo()
        _check(load().crum_image_info_get(self.handle, ctypes.byref(i)), "crum_image_info_get")
        return i.as_dict()

    def to_bytes(self) -> bytes:
        # a failed sink (EIO) leaves the drained bytes usable
        self.wait(WAIT_DRAINED, allow=(OK, ECOLLISION, EIO))
        n = self.info()["image_bytes"]
        buf = ctypes.create_string_buffer(n)
        _check(load().crum_image_copy(self.handle, buf, n), "crum_image_copy")
        return buf.raw

    def copy_into(self, dst_ptr: int, nbytes: int) -> None:
        _check(load().crum_image_copy(self.handle, dst_ptr, nbytes), "crum_image_copy")

    def save(self, path: str) -> None:
        _check(load().crum_image_save(self.handle, path.encode()), "crum_image_save")

    def release(self) -> None:
        if self.handle:
            load().crum_image_release(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class CheckpointSet:
    """A registration set on one device (``crum_set``)."""

    def __init__(self, cfg: Optional[Config] = None, **kw):
        if cfg is None:
            cfg = config(**kw)
        h = _VP()
        _check(load().crum_set_create(ctypes.byref(cfg), ctypes.byref(h)), "crum_set_create")
        self.handle = h.value

    def register(self, ptr: int, nbytes: int) -> int:
        i = _U32()
        _check(load().crum_register(self.handle, ptr, nbytes, ctypes.byref(i)), "crum_register")
        return i.value

    def unregister(self, alloc_id: int) -> None:
        _check(load().crum_unregister(self.handle, alloc_id), "crum_unregister")

    def info(self):
        a, p = _U32(), _U64()
        _check(load().crum_set_info(self.handle, ctypes.byref(a), ctypes.byref(p)), "crum_set_info")
        return a.value, p.value

    def autotune(self) -> dict:
        """Pick the fastest hash and gather mappings for the registrations."""
        hm, gm = _I(), _I()
        ht, gt = (ctypes.c_double * NUM_HASH_MAPPINGS)(), (ctypes.c_double * NUM_GATHER_MAPPINGS)()
        _check(load().crum_autotune(self.handle, ctypes.byref(hm), ctypes.byref(gm), ht, gt),
               "crum_autotune")
        return {"hash_mapping": hm.value, "gather_mapping": gm.value,
                "hash_ms": list(ht), "gather_ms": list(gt)}

    def checkpoint(self, stream: int = 0, flags: int = INCR) -> Image:
        h = _VP()
        _check(load().crum_checkpoint(self.handle, stream, flags, ctypes.byref(h)), "crum_checkpoint")
        return Image(h.value)

    def restore(self, image: Image, stream: int = 0) -> None:
        _check(load().crum_restore(self.handle, image.handle, stream), "crum_restore")

    def restore_pages(self) -> int:
        """Pages the last restore copied across the host link (waits for it)."""
        n = _U64()
        _check(load().crum_restore_pages(self.handle, ctypes.byref(n)), "crum_restore_pages")
        return n.value

    def load_image(self, path: str, parent: Optional[Image] = None) -> Image:
        h = _VP()
        _check(load().crum_image_load(self.handle, path.encode(), parent.handle if parent else None,
                                      ctypes.byref(h)), "crum_image_load")
        return Image(h.value)

    def image_from_bytes(self, data: bytes, parent: Optional[Image] = None) -> Image:
        h = _VP()
        _check(load().crum_image_from_bytes(self.handle, data, len(data),
                                            parent.handle if parent else None, ctypes.byref(h)),
               "crum_image_from_bytes")
        return Image(h.value)

    def hashes(self, n: Optional[int] = None):
        import numpy as np
        if n is None:
            n = self.info()[1]
        out = np.zeros(n, dtype=np.uint64)
        _check(load().crum_get_hashes(self.handle, out.ctypes.data, n), "crum_get_hashes")
        return out

    def poke_hash(self, page: int, value: int) -> None:
        _check(load().crum_poke_hash(self.handle, page, value), "crum_poke_hash")

    def destroy(self) -> None:
        if self.handle:
            load().crum_set_destroy(self.handle)
            self.handle = 0

    def __enter__(self) -> "CheckpointSet":
        return self

    def __exit__(self, *exc) -> None:
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Server:
    """Checkpoint/restore request server (``crum_server``)."""

    def __init__(self, device: int = 0, staging_budget: int = 16 << 30, max_inflight: int = 8,
                 max_checkpoints: int = 0, max_restores: int = 0, serialize_drains: int = 0,
                 keep_images: int = 0, order: int = 0):
        cfg = ServerConfig(device, staging_budget, max_inflight, max_checkpoints, max_restores,
                           serialize_drains, order, keep_images)
        h = _VP()
        _check(load().crum_server_create(ctypes.byref(cfg), ctypes.byref(h)), "crum_server_create")
        self.handle = h.value

    def add_client(self, cset: "CheckpointSet", stream: int) -> int:
        i = _U32()
        _check(load().crum_server_add_client(self.handle, cset.handle, stream, ctypes.byref(i)),
               "crum_server_add_client")
        return i.value

    def submit(self, client: int, kind: int = REQ_CHECKPOINT) -> int:
        rid = _U64()
        _check(load().crum_server_submit(self.handle, client, kind, ctypes.byref(rid)),
               "crum_server_submit")
        return rid.value

    def wait(self, request_id: int, stage: int = WAIT_PERSISTED, timeout_s: Optional[float] = None,
             allow=(OK, ECOLLISION)) -> dict:
        info = RequestInfo()
        t = -1 if timeout_s is None else int(timeout_s * 1e9)
        _check(load().crum_server_wait(self.handle, request_id, stage, t, ctypes.byref(info)),
               "crum_server_wait", allow)
        return info.as_dict()

    def take_image(self, request_id: int) -> Image:
        """The image of a completed checkpoint request (keep_images=1)."""
        h = _VP()
        _check(load().crum_server_take_image(self.handle, request_id, ctypes.byref(h)),
               "crum_server_take_image")
        return Image(h.value)

    def drain(self) -> dict:
        st = ServerStats()
        _check(load().crum_server_drain(self.handle, ctypes.byref(st)), "crum_server_drain")
        return st.as_dict()

    def reset_stats(self) -> None:
        _check(load().crum_server_reset_stats(self.handle), "crum_server_reset_stats")

    def destroy(self) -> None:
        if self.handle:
            load().crum_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
