"""GB300 (sm_103a) two-stage validating JSON parser -- Python binding.

Thin ctypes marshalling over the C ABI declared in include/sj.h; every step of
the parse runs in the CUDA kernels of csrc/.  PyTorch supplies device memory
and streams.  There is no CPU fallback: if the CUDA library is missing or no
GPU is present, calls raise.

    import paper_1902_08318_gb300 as sj
    p = sj.Parser(max_bytes=1 << 20)
    r = p.parse(torch_uint8_tensor_or_bytes)
    r.error, r.indices(), r.tape(), r.strings()
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libsj.so")
_SOURCES = ["api.cu", "s1.cu", "scan.cu", "s2.cu", "stage1.cu", "noalloc.cu", "server.cpp",
            "query.cu"]
_HEADERS = ["sj_internal.cuh", "s1_common.cuh", "number.cuh", "strings.cuh", "pow5_table.h"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xptxas", "-O3"]

ERROR_NAMES = ["SUCCESS", "CAPACITY", "MEMALLOC", "TAPE_ERROR", "DEPTH_ERROR", "STRING_ERROR",
               "T_ATOM_ERROR", "F_ATOM_ERROR", "N_ATOM_ERROR", "NUMBER_ERROR", "UTF8_ERROR",
               "UNCLOSED_STRING", "UNESCAPED_CHARS", "EMPTY", "INVALID_ARG", "INTERNAL"]
globals().update({name: code for code, name in enumerate(ERROR_NAMES)})

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a into _build/libsj.so (in-tree)."""
    srcs = [os.path.join(_CSRC, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_CSRC, h) for h in _HEADERS] + [os.path.join(_ROOT, "include", "sj.h")]
    with _lock:
        if (not force and os.path.exists(LIB_PATH)
                and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
            return LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        inc = ["-I", os.path.join(_ROOT, "include"), "-I", _CSRC]

        def compile_one(src):
            obj = os.path.join(_BUILD, os.path.basename(src) + ".o")
            cmd = [_nvcc(), *NVCC_FLAGS, *inc, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            subprocess.check_call(cmd)
            return obj

        with ThreadPoolExecutor(len(srcs)) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                               "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _DocResult(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("n_indices", ctypes.c_uint64), ("tape_words", ctypes.c_uint64),
                ("string_bytes", ctypes.c_uint64), ("indices_offset", ctypes.c_uint64),
                ("tape_offset", ctypes.c_uint64), ("strings_offset", ctypes.c_uint64)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_batch_bytes", ctypes.c_uint64),
                ("max_batch_docs", ctypes.c_uint32), ("max_slots", ctypes.c_uint32),
                ("max_depth", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


COMPLETION_DTYPE = np.dtype([("ticket", np.uint64), ("error", np.int32), ("slot", np.uint32),
                             ("n_indices", np.uint64), ("tape_words", np.uint64),
                             ("string_bytes", np.uint64), ("indices", np.uint64),
                             ("tape", np.uint64), ("strings", np.uint64)])


class _Result(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("n_indices", ctypes.c_uint64), ("tape_words", ctypes.c_uint64),
                ("string_bytes", ctypes.c_uint64), ("indices", ctypes.c_void_p),
                ("tape", ctypes.c_void_p), ("strings", ctypes.c_void_p)]


DOC_RESULT_DTYPE = np.dtype([("error", np.int32), ("reserved", np.uint32),
                             ("n_indices", np.uint64), ("tape_words", np.uint64),
                             ("string_bytes", np.uint64), ("indices_offset", np.uint64),
                             ("tape_offset", np.uint64), ("strings_offset", np.uint64)])


def load(path: str | None = None):
    """Load the CUDA library (no compile).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    _lib = _bind(ctypes.CDLL(path))
    return _lib


# Stage-1 variants for the measurements of "Effect of Specific Optimizations"
# (Table "tab:optimization"): each swaps one optimised step for its plain form
# (the macros are described in csrc/s1_common.cuh) and gives the same results.
ABLATIONS = {
    "prefix_xor_loop": "SJ_ABL_PREFIX_XOR_LOOP",
    "quote_parity_shfl": "SJ_ABL_QUOTE_PARITY_SHFL",
    "compare_classify": "SJ_ABL_COMPARE_CLASSIFY",
    "utf8_always": "SJ_ABL_UTF8_ALWAYS",
    "naive_flatten": "SJ_ABL_NAIVE_FLATTEN",
}
_variants = {}


def _variant_path(name: str) -> str:
    """Build (when stale) the library with stage-1 variant `name`: s1.cu
    compiled with the variant's macro, linked with the library's other
    objects into _build/variants/libsj_<name>.so."""
    macro = ABLATIONS[name]
    vdir = os.path.join(_BUILD, "variants")
    os.makedirs(vdir, exist_ok=True)
    out = os.path.join(vdir, f"libsj_{name}.so")
    deps = [os.path.join(_CSRC, f) for f in ("s1.cu", "s1_common.cuh", "sj_internal.cuh")] + [LIB_PATH]
    if os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps):
        return out
    inc = ["-I", os.path.join(_ROOT, "include"), "-I", _CSRC]
    obj = os.path.join(vdir, f"s1_{name}.o")
    subprocess.check_call([_nvcc(), *NVCC_FLAGS, *inc, f"-D{macro}", "-c",
                           os.path.join(_CSRC, "s1.cu"), "-o", obj])
    objs = [os.path.join(_BUILD, f + ".o") for f in _SOURCES if f != "s1.cu"]
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                           "-o", tmp, obj, *objs, "-lcudart"])
    os.replace(tmp, out)
    return out


def build_variants(names=None) -> list:
    """Build the variant libraries (all of ABLATIONS by default) in parallel."""
    names = list(names or ABLATIONS)
    build()
    with ThreadPoolExecutor(len(names)) as ex:
        return list(ex.map(_variant_path, names))


def load_variant(name: str):
    """The library with one stage-1 variant of ABLATIONS compiled in (built on
    first use), loaded beside the main library."""
    if name not in _variants:
        build()
        _variants[name] = _bind(ctypes.CDLL(_variant_path(name)))
    return _variants[name]


def _bind(lib):
    """Declare the argument and result types of the C ABI on a loaded library."""
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    lib.sj_parser_create.argtypes = [ctypes.POINTER(vp), u64, u32, u32]
    lib.sj_parser_create.restype = ctypes.c_int
    lib.sj_parser_destroy.argtypes = [vp]
    lib.sj_parser_destroy.restype = None
    lib.sj_parse.argtypes = [vp, vp, u64, vp, ctypes.POINTER(_Result)]
    lib.sj_parse.restype = ctypes.c_int
    lib.sj_parse_async.argtypes = [vp, vp, u64, vp]
    lib.sj_parse_async.restype = ctypes.c_int
    lib.sj_parse_wait.argtypes = [vp, ctypes.POINTER(_Result)]
    lib.sj_parse_wait.restype = ctypes.c_int
    lib.sj_parse_batch.argtypes = [vp, vp, vp, u32, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(vp)]
    lib.sj_parse_batch.restype = ctypes.c_int
    lib.sj_parser_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.sj_parser_set_profiling.restype = ctypes.c_int
    lib.sj_parser_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.sj_parser_stage_times.restype = ctypes.c_int
    lib.sj_parser_kernels_per_run.argtypes = [vp]
    lib.sj_parser_kernels_per_run.restype = ctypes.c_int
    lib.sj_parser_prepare.argtypes = [vp, u32]
    lib.sj_parser_prepare.restype = ctypes.c_int
    lib.sj_parser_set_host_chunk.argtypes = [vp, u64]
    lib.sj_parser_set_host_chunk.restype = ctypes.c_int
    lib.sj_stage1_indices_noalloc.argtypes = [vp, u64, vp, vp, vp]
    lib.sj_stage1_indices_noalloc.restype = ctypes.c_int
    lib.sj_error_name.argtypes = [ctypes.c_int]
    lib.sj_error_name.restype = ctypes.c_char_p
    lib.sj_last_cuda_error.argtypes = []
    lib.sj_last_cuda_error.restype = ctypes.c_int
    lib.sj_version.argtypes = []
    lib.sj_version.restype = ctypes.c_char_p
    lib.sj_parse_batch_async.argtypes = [vp, vp, vp, u32, vp]
    lib.sj_parse_batch_async.restype = ctypes.c_int
    lib.sj_parse_query.argtypes = [vp]
    lib.sj_parse_query.restype = ctypes.c_int
    lib.sj_parse_batch_wait.argtypes = [vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(vp)]
    lib.sj_parse_batch_wait.restype = ctypes.c_int
    lib.sj_query_create.argtypes = [ctypes.POINTER(vp), u64]
    lib.sj_query_create.restype = ctypes.c_int
    lib.sj_query_destroy.argtypes = [vp]
    lib.sj_query_destroy.restype = None
    lib.sj_query_distinct.argtypes = [vp, vp, u64, vp, u64, vp, u32, vp, ctypes.POINTER(u64),
                                      ctypes.POINTER(vp)]
    lib.sj_query_distinct.restype = ctypes.c_int
    lib.sj_parser_get_launch.argtypes = [vp, vp, vp]
    lib.sj_parser_get_launch.restype = ctypes.c_int
    lib.sj_parser_set_launch.argtypes = [vp, vp]
    lib.sj_parser_set_launch.restype = ctypes.c_int
    lib.sj_parser_autotune.argtypes = [vp, vp, u64, vp, ctypes.c_int, vp, vp]
    lib.sj_parser_autotune.restype = ctypes.c_int
    lib.sj_parser_device_bytes.argtypes = [vp]
    lib.sj_parser_device_bytes.restype = u64
    lib.sj_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_ServerConfig)]
    lib.sj_server_create.restype = ctypes.c_int
    lib.sj_server_destroy.argtypes = [vp]
    lib.sj_server_destroy.restype = None
    lib.sj_server_slots.argtypes = [vp]
    lib.sj_server_slots.restype = u32
    lib.sj_server_device_bytes.argtypes = [vp]
    lib.sj_server_device_bytes.restype = u64
    lib.sj_server_batches.argtypes = [vp]
    lib.sj_server_batches.restype = u64
    lib.sj_server_submit.argtypes = [vp, vp, u64, ctypes.POINTER(u64)]
    lib.sj_server_submit.restype = ctypes.c_int
    lib.sj_server_poll.argtypes = [vp, vp, u32]
    lib.sj_server_poll.restype = ctypes.c_int
    lib.sj_server_release.argtypes = [vp, u64]
    lib.sj_server_release.restype = ctypes.c_int
    lib.sj_server_replay.argtypes = [vp, vp, vp, vp, u32, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sj_server_replay.restype = ctypes.c_int
    return lib


EXPORTED = ["sj_parser_create", "sj_parser_destroy", "sj_parse", "sj_parse_async", "sj_parse_wait",
            "sj_parse_batch", "sj_parser_set_profiling", "sj_parser_stage_times",
            "sj_parser_kernels_per_run", "sj_stage1_indices_noalloc", "sj_error_name",
            "sj_last_cuda_error", "sj_version", "sj_parse_batch_async", "sj_parse_query",
            "sj_parse_batch_wait", "sj_parser_device_bytes", "sj_server_create",
            "sj_server_destroy", "sj_server_slots", "sj_server_device_bytes", "sj_server_batches",
            "sj_server_submit", "sj_server_poll", "sj_server_release", "sj_server_replay",
            "sj_parser_get_launch", "sj_parser_set_launch", "sj_parser_autotune",
            "sj_query_create", "sj_query_destroy", "sj_query_distinct",
            "sj_parser_set_host_chunk", "sj_parser_prepare"]
TUNED_KERNELS = ("s1_blocks", "s1_flatten", "s2_reduce", "s2_build")
STAGES = ("setup", "s1_blocks", "s1_scan", "s1_flatten", "s2_reduce", "s2_scan_frontier",
          "s2_numbers", "s2_build", "finalize")


class SJError(RuntimeError):
    pass


def _check(status: int):
    if status != 0:
        lib = load()
        raise SJError(f"sj call failed: {ERROR_NAMES[status] if status < 16 else status}"
                      f" (cuda error {lib.sj_last_cuda_error()})")


class _DeviceView:
    """__cuda_array_interface__ over parser-owned device memory (no copy)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _device_tensor(ptr: int, n: int, typestr: str):
    import torch
    return torch.as_tensor(_DeviceView(ptr, n, typestr), device="cuda")


def _as_input(data):
    """(pointer, length, keepalive) of a torch tensor (device or host), numpy array or bytes."""
    try:
        import torch
        if isinstance(data, torch.Tensor):
            t = data.contiguous()
            if t.dtype != torch.uint8:
                t = t.view(torch.uint8)
            return t.data_ptr(), t.numel(), t
    except ImportError:
        pass
    if isinstance(data, (bytes, bytearray, memoryview)):
        a = np.frombuffer(bytes(data), dtype=np.uint8)
    else:
        a = np.ascontiguousarray(data, dtype=np.uint8)
    return a.ctypes.data, a.size, a


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Result:
    """One document's result.  Accessors return device tensors (views)."""

    def __init__(self, error, n_indices, tape_words, string_bytes, idx_ptr, tape_ptr, str_ptr):
        self.error = int(error)
        self.error_name = ERROR_NAMES[self.error]
        self.n_indices = int(n_indices)
        self.tape_words = int(tape_words)
        self.string_bytes = int(string_bytes)
        self._p = (idx_ptr, tape_ptr, str_ptr)

    def indices(self):
        return _device_tensor(self._p[0], self.n_indices, "<u4")

    def tape(self):
        return _device_tensor(self._p[1], self.tape_words, "<u8")

    def strings(self):
        return _device_tensor(self._p[2], self.string_bytes, "|u1")


class Parser:
    """A parser owning device buffers for inputs up to max_bytes (summed over a
    batch) and max_docs documents per batch."""

    def __init__(self, max_bytes: int, max_docs: int = 1, max_depth: int = 0, lib=None):
        import torch
        if not torch.cuda.is_available():
            raise SJError("no CUDA device: the parser has no CPU path")
        self._lib = lib if lib is not None else load()
        h = ctypes.c_void_p()
        _check(self._lib.sj_parser_create(ctypes.byref(h), int(max_bytes), int(max_docs),
                                          int(max_depth)))
        self._h = h
        self.max_bytes = int(max_bytes)
        self.max_docs = int(max_docs)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sj_parser_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def parse(self, data, stream=None) -> Result:
        ptr, n, keep = _as_input(data)
        r = _Result()
        _check(self._lib.sj_parse(self._h, ptr, n, _stream_handle(stream), ctypes.byref(r)))
        del keep
        return Result(r.error, r.n_indices, r.tape_words, r.string_bytes, r.indices, r.tape,
                      r.strings)

    def parse_async(self, data, stream=None):
        ptr, n, keep = _as_input(data)
        _check(self._lib.sj_parse_async(self._h, ptr, n, _stream_handle(stream)))
        return keep

    def parse_wait(self) -> Result:
        r = _Result()
        _check(self._lib.sj_parse_wait(self._h, ctypes.byref(r)))
        return Result(r.error, r.n_indices, r.tape_words, r.string_bytes, r.indices, r.tape,
                      r.strings)

    def parse_batch(self, data, offsets, stream=None):
        """Returns (results: structured numpy array, indices, tape, strings device tensors
        covering the batch output arrays)."""
        ptr, n, keep = _as_input(data)
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        nd = off.size - 1
        out = np.zeros(nd, dtype=DOC_RESULT_DTYPE)
        pi, pt, ps = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(self._lib.sj_parse_batch(self._h, ptr, off.ctypes.data, nd, _stream_handle(stream),
                                        out.ctypes.data, ctypes.byref(pi), ctypes.byref(pt),
                                        ctypes.byref(ps)))
        del keep
        return out, (pi.value, pt.value, ps.value)

    def set_profiling(self, on: bool):
        _check(self._lib.sj_parser_set_profiling(self._h, int(bool(on))))

    def stage_times(self) -> dict:
        """Kernel durations (ms) of the last run, measured with CUDA events on
        its stream (profiling must be on)."""
        ms = (ctypes.c_float * len(STAGES))()
        _check(self._lib.sj_parser_stage_times(self._h, ms, len(STAGES)))
        return dict(zip(STAGES, [float(x) for x in ms]))

    def kernels_per_run(self) -> int:
        return int(self._lib.sj_parser_kernels_per_run(self._h))

    def prepare(self, max_docs: int = 0):
        """Capture the runs of every batch size up to max_docs now."""
        _check(self._lib.sj_parser_prepare(self._h, int(max_docs)))

    def set_host_chunk(self, chunk_bytes: int):
        """Chunk size for single documents in pinned host memory, parsed while
        they are copied (0: never chunk)."""
        _check(self._lib.sj_parser_set_host_chunk(self._h, int(chunk_bytes)))

    @staticmethod
    def view(ptr: int, n: int, typestr: str):
        return _device_tensor(ptr, n, typestr)

    def device_bytes(self) -> int:
        return int(self._lib.sj_parser_device_bytes(self._h))

    def launch(self) -> dict:
        """Resident blocks per SM of the four main kernels, and their limits."""
        cur = np.zeros(4, dtype=np.uint32)
        lim = np.zeros(4, dtype=np.uint32)
        _check(self._lib.sj_parser_get_launch(self._h, cur.ctypes.data, lim.ctypes.data))
        return {k: (int(c), int(m)) for k, c, m in zip(TUNED_KERNELS, cur, lim)}

    def set_launch(self, blocks_per_sm):
        b = np.ascontiguousarray(blocks_per_sm, dtype=np.uint32)
        _check(self._lib.sj_parser_set_launch(self._h, b.ctypes.data))

    def autotune(self, sample, stream=None, reps: int = 2) -> dict:
        """Pick each main kernel's blocks per SM by timing it on `sample`."""
        ptr, n, keep = _as_input(sample)
        bps = np.zeros(4, dtype=np.uint32)
        ms = np.zeros(4, dtype=np.float32)
        _check(self._lib.sj_parser_autotune(self._h, ptr, n, _stream_handle(stream), int(reps),
                                            bps.ctypes.data, ms.ctypes.data))
        del keep
        return {k: {"blocks_per_sm": int(b), "ms": round(float(t), 4)}
                for k, b, t in zip(TUNED_KERNELS, bps, ms)}


class Server:
    """Continuous-batching parse server (sj_server_* of include/sj.h).

    submit() queues host bytes (kept alive here until the request's batch is
    formed); poll() launches waiting requests on free slots and returns the
    finished ones as a COMPLETION_DTYPE array, whose pointers stay valid until
    release(ticket)."""

    def __init__(self, max_batch_bytes: int = 16 << 20, max_batch_docs: int = 4096,
                 max_slots: int = 8, mem_budget: int = 8 << 30, max_depth: int = 0):
        self._lib = load()
        cfg = _ServerConfig(int(mem_budget), int(max_batch_bytes), int(max_batch_docs),
                            int(max_slots), int(max_depth), 0)
        h = ctypes.c_void_p()
        _check(self._lib.sj_server_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h
        self._keep = {}
        self._buf = np.zeros(1024, dtype=COMPLETION_DTYPE)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sj_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def slots(self) -> int:
        return int(self._lib.sj_server_slots(self._h))

    @property
    def device_bytes(self) -> int:
        return int(self._lib.sj_server_device_bytes(self._h))

    @property
    def batches(self) -> int:
        return int(self._lib.sj_server_batches(self._h))

    def submit(self, data) -> int:
        b = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8) if isinstance(data, (bytes, bytearray))
                                 else data, dtype=np.uint8)
        t = ctypes.c_uint64()
        _check(self._lib.sj_server_submit(self._h, b.ctypes.data if b.size else None, b.size,
                                          ctypes.byref(t)))
        self._keep[t.value] = b
        return t.value

    def poll(self) -> np.ndarray:
        n = self._lib.sj_server_poll(self._h, self._buf.ctypes.data, self._buf.size)
        if n < 0:
            _check(-n)
        out = self._buf[:n].copy()
        for tk in out["ticket"]:
            self._keep.pop(int(tk), None)
        return out

    def release(self, ticket: int):
        _check(self._lib.sj_server_release(self._h, int(ticket)))

    def replay(self, buf: np.ndarray, offsets: np.ndarray, arrival_s: np.ndarray):
        """Replay an arrival trace natively; returns (latency_s array, wall seconds)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        n = arr.size
        lat = np.zeros(n, dtype=np.float64)
        wall = ctypes.c_double()
        _check(self._lib.sj_server_replay(self._h, buf.ctypes.data, off.ctypes.data,
                                          arr.ctypes.data, n, lat.ctypes.data,
                                          ctypes.byref(wall)))
        return lat, wall.value


class Query:
    """Distinct int64 values at a key path over a parsed document's device
    tape (sj_query_* of include/sj.h): the paper's user.id query."""

    def __init__(self, max_values: int = 1 << 20):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.sj_query_create(ctypes.byref(h), int(max_values)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sj_query_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def distinct(self, result, path, stream=None):
        """result: a successful Result of Parser.parse; path: e.g. ("user", "id").
        Returns a device tensor (int64) of the distinct values."""
        keys = [k.encode() for k in path]
        arr = (ctypes.c_char_p * len(keys))(*keys)
        n = ctypes.c_uint64()
        vals = ctypes.c_void_p()
        _check(self._lib.sj_query_distinct(self._h, result._p[1], result.tape_words,
                                           result._p[2], result.string_bytes, arr, len(keys),
                                           _stream_handle(stream), ctypes.byref(n),
                                           ctypes.byref(vals)))
        return _device_tensor(vals.value, n.value, "<i8")
