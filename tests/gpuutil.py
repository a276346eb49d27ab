"""Helpers for the GPU parity tests: run the CUDA library through its C ABI
(the ctypes binding) and compare with the oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle

NO_INDEX_COMPARE = (oracle.UTF8_ERROR, oracle.CAPACITY, oracle.EMPTY)


def gpu_result(parser, doc, stream=None) -> dict:
    import torch
    r = parser.parse(doc, stream=stream)
    out = {"error": r.error, "n_indices": r.n_indices}
    torch.cuda.synchronize()
    out["indices"] = r.indices().cpu().numpy().copy() if r.n_indices else np.zeros(0, np.uint32)
    if r.error == 0:
        out["tape"] = r.tape().cpu().numpy().copy()
        out["strings"] = r.strings().cpu().numpy().copy()
    return out


def compare(got: dict, exp: dict, label=""):
    assert got["error"] == exp["error"], (
        f"{label}: error {oracle_name(got['error'])} != oracle {oracle_name(exp['error'])}")
    if exp["error"] not in NO_INDEX_COMPARE:
        assert got["n_indices"] == exp["n_indices"], f"{label}: n_indices"
        gi, ei = got["indices"], exp["indices"]
        if not np.array_equal(gi, ei):
            bad = np.nonzero(gi[: min(len(gi), len(ei))] != ei[: min(len(gi), len(ei))])[0]
            raise AssertionError(f"{label}: indices differ first at {bad[:5]}")
    if exp["error"] == 0:
        gt, et = got["tape"], exp["tape"]
        assert gt.size == et.size, f"{label}: tape size {gt.size} != {et.size}"
        if not np.array_equal(gt, et):
            bad = np.nonzero(gt != et)[0]
            raise AssertionError(f"{label}: tape differs at {bad[:5]} got {gt[bad[:3]]} exp {et[bad[:3]]}")
        gs, es = got["strings"], exp["strings"]
        assert gs.size == es.size, f"{label}: strings size {gs.size} != {es.size}"
        assert np.array_equal(gs, es), f"{label}: strings differ at {np.nonzero(gs != es)[0][:5]}"


def oracle_name(code: int) -> str:
    names = ["SUCCESS", "CAPACITY", "MEMALLOC", "TAPE_ERROR", "DEPTH_ERROR", "STRING_ERROR",
             "T_ATOM_ERROR", "F_ATOM_ERROR", "N_ATOM_ERROR", "NUMBER_ERROR", "UTF8_ERROR",
             "UNCLOSED_STRING", "UNESCAPED_CHARS", "EMPTY", "INVALID_ARG", "INTERNAL"]
    return names[code] if 0 <= code < len(names) else str(code)


def check_doc(parser, doc, label="", max_depth=0):
    b = doc if isinstance(doc, (bytes, bytearray)) else np.asarray(doc, dtype=np.uint8).tobytes()
    exp = oracle.parse(b, max_depth=max_depth)
    got = gpu_result(parser, np.frombuffer(b, dtype=np.uint8))
    compare(got, exp, label or repr(b[:40]))
    return got


def batch_arrays(docs):
    lens = np.array([len(d) for d in docs], dtype=np.uint64)
    off = np.zeros(len(docs) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    buf = np.frombuffer(b"".join(docs), dtype=np.uint8) if docs else np.zeros(0, np.uint8)
    return buf, off


def batch_outputs(parser, res, ptrs, total_bytes, n_docs):
    """Copy the batch output arrays to the host."""
    import torch
    pi, pt, ps = ptrs
    idx = parser.view(pi, total_bytes + 16, "<u4").cpu().numpy()
    tape = parser.view(pt, total_bytes + 3 * n_docs + 8, "<u8").cpu().numpy()
    strs = parser.view(ps, (5 * total_bytes) // 2 + 8 * n_docs + 64, "|u1").cpu().numpy()
    torch.cuda.synchronize()
    return idx, tape, strs


def compare_batch_doc(res_i, outs, exp, label):
    idx, tape, strs = outs
    got = {"error": int(res_i["error"]), "n_indices": int(res_i["n_indices"])}
    io, to, so = int(res_i["indices_offset"]), int(res_i["tape_offset"]), int(res_i["strings_offset"])
    got["indices"] = idx[io: io + got["n_indices"]]
    if got["error"] == 0:
        got["tape"] = tape[to: to + int(res_i["tape_words"])]
        got["strings"] = strs[so: so + int(res_i["string_bytes"])]
    compare(got, exp, label)
