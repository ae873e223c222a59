"""Python binding of the PGCP CUDA library (argument marshalling only).

Every computation runs in libpgcp.so (include/pgcp.h); this module converts
torch tensors / numpy arrays into pointers and sizes, passes the current CUDA
stream, and raises ``PgcpError`` on a non-zero status.  Importing it loads the
library and raises if it is missing or was built for another machine.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpgcp.so")
METRICS_NOALLOC_MAX_FACES = 262144   # PGCP_METRICS_NOALLOC_MAX_FACES

FREE, DISK, SPHERE = 0, 1, 2
FP64, FP32_REFINED, DF64_REFINED = 0, 1, 2
WARM_COLD, WARM_WELDMAP, WARM_LEARNED = 0, 1, 2
# parameter layout of the learned warm-start network (pgcp.h): matrices rows = inputs
GNN_PARAM_SHAPES = [(16, 64), (64,)] + [(128, 64), (64,)] * 4 + [(64, 16), (16,)]

STATUS = {0: "OK", 1: "ARG", 2: "CUDA", 3: "OOM", 4: "NONMANIFOLD", 5: "TOPOLOGY", 6: "SCHEDULE",
          7: "DEGENERATE", 8: "NO_CONVERGENCE", 9: "NUMERIC"}


class PgcpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.code = STATUS.get(status, str(status))


class Options(C.Structure):
    _fields_ = [("variant", C.c_int32), ("precision", C.c_int32), ("tol", C.c_double), ("max_iters", C.c_int32),
                ("max_refine", C.c_int32), ("inner_tol", C.c_double), ("warm_start", C.c_int32),
                ("interior_map_fp64", C.c_int32), ("block_rows_log2", C.c_int32), ("local_precision", C.c_int32),
                ("spmv_lanes", C.c_int32), ("pcg_blocks_per_sm", C.c_int32),
                ("pcg_schedule", C.c_int32), ("deterministic", C.c_int32), ("local_precond", C.c_int32),
                ("reserved", C.c_int32 * 1)]


class Stats(C.Structure):
    _fields_ = [("K", C.c_int32), ("n_welds", C.c_int32), ("dncp_iters", C.c_int32), ("final_iters", C.c_int32),
                ("dncp_refine", C.c_int32), ("final_refine", C.c_int32), ("dncp_relres", C.c_double),
                ("final_relres", C.c_double), ("seam_mismatch", C.c_double), ("ms_partition", C.c_double),
                ("ms_assembly", C.c_double), ("ms_local", C.c_double), ("ms_weld", C.c_double),
                ("ms_final", C.c_double), ("nnz", C.c_int64), ("n_copies", C.c_int64), ("pcg_ms", C.c_double),
                ("pcg_bytes", C.c_double), ("pcg_launches", C.c_int32), ("learned_pieces", C.c_int32),
                ("pcg_bytes_touched", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Distortion(C.Structure):
    _fields_ = [("mean", C.c_double), ("sd", C.c_double), ("median", C.c_double), ("iqr", C.c_double),
                ("max", C.c_double), ("n_corners", C.c_int64), ("flips", C.c_int64), ("max_mu", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FoldReport(C.Structure):
    _fields_ = [("folded_before", C.c_int64), ("folded_after", C.c_int64), ("rounds", C.c_int32),
                ("pieces_fixed", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AreaResult(C.Structure):
    _fields_ = [("param", C.c_double * 3), ("before", C.c_double), ("after", C.c_double),
                ("evals", C.c_int32), ("status", C.c_int32)]

    def as_dict(self):
        """param: complex alpha or q (planar); param3: the three stored values (a for the sphere)."""
        return {"param": complex(self.param[0], self.param[1]), "param3": list(self.param),
                "before": self.before, "after": self.after, "evals": self.evals,
                "status": STATUS.get(self.status, str(self.status))}


# exported symbols and their signatures (name -> (restype, argtypes))
_P = C.c_void_p
SIGNATURES = {
    "pgcp_default_options": (None, [C.POINTER(Options)]),
    "pgcp_create": (C.c_int, [C.POINTER(_P), C.POINTER(Options), _P]),
    "pgcp_destroy": (C.c_int, [_P]),
    "pgcp_set_options": (C.c_int, [_P, C.POINTER(Options)]),
    "pgcp_last_error": (C.c_char_p, [_P]),
    "pgcp_status_string": (C.c_char_p, [C.c_int]),
    "pgcp_launch_count": (C.c_int64, []),
    "pgcp_alloc_count": (C.c_int64, []),
    "pgcp_partition": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P, C.c_int32, C.c_int32,
                                 C.POINTER(_P)]),
    "pgcp_partition_batch": (C.c_int, [_P, C.c_int32, C.POINTER(_P), C.POINTER(C.c_int64), C.POINTER(_P),
                                       C.POINTER(C.c_int64), C.POINTER(_P), C.c_int32, C.c_int32, C.POINTER(_P)]),
    "pgcp_part_free": (C.c_int, [_P]),
    "pgcp_part_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "pgcp_part_info": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pgcp_part_get_partition": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "pgcp_local_param": (C.c_int, [_P, _P]),
    "pgcp_part_get_csr": (C.c_int, [_P, _P, _P, _P, _P]),
    "pgcp_part_get_coords": (C.c_int, [_P, _P, C.c_int32, _P]),
    "pgcp_weld": (C.c_int, [_P, _P]),
    "pgcp_global_solve": (C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(Stats)]),
    "pgcp_metrics": (C.c_int, [_P, _P, _P, C.POINTER(Distortion)]),
    "pgcp_metrics_noalloc": (C.c_int, [_P, _P, _P, C.POINTER(Distortion)]),
    "pgcp_area_distortion": (C.c_int, [_P, _P, _P, C.POINTER(C.c_double)]),
    "pgcp_area_mobius": (C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(AreaResult)]),
    "pgcp_fix_folds": (C.c_int, [_P, _P, _P, C.POINTER(FoldReport)]),
    "pgcp_set_piece_mask": (C.c_int, [_P, _P, _P]),
    "pgcp_part_get_boundary": (C.c_int, [_P, _P, C.c_int32, _P]),
    "pgcp_part_set_boundary": (C.c_int, [_P, _P, C.c_int32, _P]),
    "pgcp_run": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P, C.c_int32, _P,
                           C.POINTER(Stats)]),
    "pgcp_selftest_sort": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32]),
    "pgcp_selftest_scan": (C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "pgcp_selftest_gemm_bf16": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_int64, _P, _P]),
    "pgcp_autotune": (C.c_int, [_P, _P, C.c_int32, C.POINTER(Options), C.POINTER(C.c_double)]),
    "pgcp_free_boundary": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P, _P, C.POINTER(Stats)]),
    "pgcp_disk": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P, _P, C.POINTER(Stats)]),
    "pgcp_sphere": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, _P, _P, C.POINTER(Stats)]),
    "pgcp_batch_run": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.POINTER(Stats)]),
    "pgcp_part_mesh_status": (C.c_int, [_P, _P]),
    "pgcp_gnn_num_params": (C.c_int64, []),
    "pgcp_gnn_create": (C.c_int, [_P, _P, C.POINTER(C.c_void_p)]),
    "pgcp_gnn_load": (C.c_int, [_P, C.c_char_p, C.POINTER(C.c_void_p)]),
    "pgcp_gnn_free": (C.c_int, [_P]),
    "pgcp_gnn_get_params": (C.c_int, [_P, _P, _P]),
    "pgcp_gnn_set_params": (C.c_int, [_P, _P, _P]),
    "pgcp_set_gnn": (C.c_int, [_P, _P]),
    "pgcp_gnn_inputs": (C.c_int, [_P, _P, _P, _P, _P]),
    "pgcp_gnn_grad": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_double)]),
    "pgcp_gnn_train_step": (C.c_int, [_P, _P, _P, C.c_float, C.POINTER(C.c_double)]),
    "pgcp_gnn_predict": (C.c_int, [_P, _P, _P, _P]),
    "pgcp_selftest_umma_desc": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint32]),
    "pgcp_selftest_umma_idesc": (C.c_uint32, [C.c_int32, C.c_int32]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpgcp.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_1903_12359_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().pgcp_launch_count())


def alloc_count() -> int:
    """Device allocations the library has requested so far in this process."""
    return int(load().pgcp_alloc_count())


def default_options(**kw) -> Options:
    o = Options()
    load().pgcp_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def check_coords(U, nv: int, closed: bool, device=None, inplace: bool = False):
    """Refuse, before any launch, a coordinate tensor the kernels cannot read
    safely: it must be a float64 tensor of shape (nv, 3) for a closed part and
    (nv, 2) otherwise, on the CUDA device the context is bound to (and
    contiguous when it is updated in place)."""
    dim = 3 if closed else 2
    if not isinstance(U, torch.Tensor):
        raise ValueError("coordinates must be a torch tensor")
    if U.dtype != torch.float64:
        raise ValueError(f"coordinates must be float64, got {U.dtype}")
    if tuple(U.shape) != (nv, dim):
        raise ValueError(f"coordinates must have shape ({nv}, {dim}), got {tuple(U.shape)}")
    if not U.is_cuda:
        raise ValueError("coordinates must be a CUDA tensor")
    if device is not None and U.device.index != device:
        raise ValueError(f"coordinates are on cuda:{U.device.index}, the context on cuda:{device}")
    if inplace and not U.is_contiguous():
        raise ValueError("coordinates updated in place must be contiguous")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    return t.ctypes.data_as(C.c_void_p)


def _dev(a, dtype):
    """A contiguous CUDA tensor of dtype from a numpy array or tensor."""
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


class Context:
    """A library context bound to the current device and a CUDA stream."""

    def __init__(self, options: Options | None = None, stream: torch.cuda.Stream | None = None, **kw):
        lib = load()
        self.options = options if options is not None else default_options(**kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.cuda.current_device()
        h = C.c_void_p()
        st = lib.pgcp_create(C.byref(h), C.byref(self.options), C.c_void_p(self.stream.cuda_stream))
        if st:
            raise PgcpError(st, "pgcp_create failed")
        self.h = h

    def check(self, st):
        if st:
            raise PgcpError(st, load().pgcp_last_error(self.h).decode())

    def selftest_gemm_bf16(self, A, Bt, epilogue=0, bias=None):
        """C = epi(A . Bt^T) on the tensor cores; A [M, K], Bt [N, K] bf16 CUDA tensors."""
        M, K = A.shape
        N = Bt.shape[0]
        dt = torch.bfloat16 if epilogue == 1 else torch.float32
        C_ = torch.empty((M, N), dtype=dt, device="cuda")
        self.check(load().pgcp_selftest_gemm_bf16(self.h, epilogue, N, K, _ptr(A.contiguous()), _ptr(Bt.contiguous()),
                                                  M, _ptr(bias), _ptr(C_)))
        return C_

    def autotune(self, part, probe_iters: int = 200):
        """Pick the fastest PCG schedule on `part` (pgcp_autotune); returns
        (chosen options as a dict of the tuned fields, ms per iteration)."""
        o = Options()
        ms = C.c_double()
        self.check(load().pgcp_autotune(self.h, part.h, probe_iters, C.byref(o), C.byref(ms)))
        self.options = o
        keys = ("pcg_blocks_per_sm", "pcg_schedule", "spmv_lanes", "block_rows_log2")
        return {k: getattr(o, k) for k in keys}, ms.value

    def set_gnn(self, gnn):
        """Network for warm_start = WARM_LEARNED (None detaches)."""
        self._gnn = gnn
        self.check(load().pgcp_set_gnn(self.h, None if gnn is None else gnn.h))

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self.check(load().pgcp_set_options(self.h, C.byref(self.options)))

    def close(self):
        if getattr(self, "h", None):
            load().pgcp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- primitives (self tests)
    def selftest_sort(self, keys: torch.Tensor, vals: torch.Tensor, bits: int):
        self.check(load().pgcp_selftest_sort(self.h, _ptr(keys), _ptr(vals), keys.numel(), bits))

    def selftest_scan(self, x: torch.Tensor):
        out = torch.empty(x.numel(), dtype=torch.int64, device="cuda")
        tot = C.c_int64()
        self.check(load().pgcp_selftest_scan(self.h, _ptr(x), _ptr(out), x.numel(), C.byref(tot)))
        return out, tot.value

    # ---- stages
    def partition(self, V, F, cut_edges=None, face_labels=None, closed=False) -> "Part":
        Vd = _dev(V, torch.float64)
        Fd = _dev(F, torch.int32)
        cd = _dev(cut_edges, torch.int32) if cut_edges is not None and len(cut_edges) else None
        ld = _dev(face_labels, torch.int32) if face_labels is not None else None
        out = C.c_void_p()
        self.check(load().pgcp_partition(self.h, _ptr(Vd), Vd.shape[0], _ptr(Fd), Fd.shape[0], _ptr(cd),
                                         0 if cd is None else cd.shape[0], _ptr(ld), 0, int(closed), C.byref(out)))
        return Part(self, out, nv=Vd.shape[0], nf=Fd.shape[0], closed=closed)

    def partition_batch(self, meshes, closed=False) -> "Part":
        """meshes: list of (V, F, face_labels)."""
        Vs = [_dev(m[0], torch.float64) for m in meshes]
        Fs = [_dev(m[1], torch.int32) for m in meshes]
        Ls = [_dev(m[2], torch.int32) for m in meshes]
        n = len(meshes)
        arrV = (C.c_void_p * n)(*[t.data_ptr() for t in Vs])
        arrF = (C.c_void_p * n)(*[t.data_ptr() for t in Fs])
        arrL = (C.c_void_p * n)(*[t.data_ptr() for t in Ls])
        nv = (C.c_int64 * n)(*[t.shape[0] for t in Vs])
        nf = (C.c_int64 * n)(*[t.shape[0] for t in Fs])
        out = C.c_void_p()
        self.check(load().pgcp_partition_batch(self.h, n, arrV, nv, arrF, nf, arrL, 0, int(closed), C.byref(out)))
        return Part(self, out, nv=sum(t.shape[0] for t in Vs), nf=sum(t.shape[0] for t in Fs), closed=closed,
                    keep=(Vs, Fs, Ls))

    def run(self, V, F, cut_edges=None, face_labels=None, host=True):
        """One-shot pipeline.  host=True: numpy in, numpy out (copies inside the call)."""
        dim = 3 if self.options.variant == SPHERE else 2
        st = Stats()
        if host:
            Vh = np.ascontiguousarray(V, dtype=np.float64)
            Fh = np.ascontiguousarray(F, dtype=np.int32)
            ch = None if cut_edges is None else np.ascontiguousarray(cut_edges, dtype=np.int32)
            lh = None if face_labels is None else np.ascontiguousarray(face_labels, dtype=np.int32)
            out = np.empty((Vh.shape[0], dim), dtype=np.float64)
            self.check(load().pgcp_run(self.h, _ptr(Vh), Vh.shape[0], _ptr(Fh), Fh.shape[0], _ptr(ch),
                                       0 if ch is None else ch.shape[0], _ptr(lh), 1, _ptr(out), C.byref(st)))
            return out, st.as_dict()
        Vd, Fd = _dev(V, torch.float64), _dev(F, torch.int32)
        cd = None if cut_edges is None else _dev(cut_edges, torch.int32)
        ld = None if face_labels is None else _dev(face_labels, torch.int32)
        out = torch.empty((Vd.shape[0], dim), dtype=torch.float64, device="cuda")
        self.check(load().pgcp_run(self.h, _ptr(Vd), Vd.shape[0], _ptr(Fd), Fd.shape[0], _ptr(cd),
                                   0 if cd is None else cd.shape[0], _ptr(ld), 0, _ptr(out), C.byref(st)))
        return out, st.as_dict()


class MeshDesc(C.Structure):
    _fields_ = [("V", C.c_void_p), ("nv", C.c_int64), ("F", C.c_void_p), ("nf", C.c_int64),
                ("face_labels", C.c_void_p)]


def one_call(ctx: "Context", variant: str, V, F, cut_edges=None, face_labels=None):
    """pgcp_free_boundary / pgcp_disk / pgcp_sphere on device copies of the inputs;
    returns (map tensor, stats dict)."""
    fn = {"free": "pgcp_free_boundary", "disk": "pgcp_disk", "sphere": "pgcp_sphere"}[variant]
    Vd, Fd = _dev(V, torch.float64), _dev(F, torch.int32)
    cd = None if cut_edges is None else _dev(cut_edges, torch.int32)
    ld = None if face_labels is None else _dev(face_labels, torch.int32)
    out = torch.empty((Vd.shape[0], 3 if variant == "sphere" else 2), dtype=torch.float64, device="cuda")
    st = Stats()
    ctx.check(getattr(load(), fn)(ctx.h, _ptr(Vd), Vd.shape[0], _ptr(Fd), Fd.shape[0], _ptr(cd),
                                  0 if cd is None else cd.shape[0], _ptr(ld), _ptr(out), C.byref(st)))
    return out, st.as_dict()


def batch_run(ctx: "Context", meshes):
    """pgcp_batch_run on [(V, F, face_labels)]: (list of map tensors, list of status names, stats)."""
    keep = [(_dev(m[0], torch.float64), _dev(m[1], torch.int32), _dev(m[2], torch.int32)) for m in meshes]
    dim = 3 if ctx.options.variant == SPHERE else 2
    outs = [torch.empty((v.shape[0], dim), dtype=torch.float64, device="cuda") for v, _, _ in keep]
    descs = (MeshDesc * len(keep))(*[MeshDesc(v.data_ptr(), v.shape[0], f.data_ptr(), f.shape[0], l.data_ptr())
                                     for v, f, l in keep])
    ptrs = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    status = (C.c_int32 * len(keep))()
    st = Stats()
    ctx.check(load().pgcp_batch_run(ctx.h, len(keep), descs, ptrs, status, C.byref(st)))
    return outs, [STATUS.get(v, str(v)) for v in status], st.as_dict()


class Part:
    def __init__(self, ctx: Context, h, nv, nf, closed, keep=None):
        self.ctx, self.h, self.nv, self.nf, self.closed = ctx, h, nv, nf, closed
        self._keep = keep
        self.stats = None

    def info(self):
        K, nc, nnz, nl, nw, nm = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        self.ctx.check(load().pgcp_part_info(self.h, C.byref(K), C.byref(nc), C.byref(nnz), C.byref(nl),
                                             C.byref(nw), C.byref(nm)))
        return {"K": K.value, "n_copies": nc.value, "nnz": nnz.value, "n_loop": nl.value, "n_welds": nw.value,
                "n_mesh": nm.value}

    def mesh_status(self):
        """Per-mesh status codes of a batch (names from STATUS)."""
        n = self.info()["n_mesh"]
        st = (C.c_int32 * n)()
        load().pgcp_part_mesh_status(self.h, st)
        return [STATUS.get(v, str(v)) for v in st]

    def get_stats(self):
        st = Stats()
        self.ctx.check(load().pgcp_part_get_stats(self.h, C.byref(st)))
        return st.as_dict()

    def partition_arrays(self):
        i = self.info()
        d = "cuda"
        fl = torch.empty(self.nf, dtype=torch.int32, device=d)
        voff = torch.empty(i["K"] + 1, dtype=torch.int64, device=d)
        verts = torch.empty(i["n_copies"], dtype=torch.int32, device=d)
        loff = torch.empty(i["K"] + 1, dtype=torch.int64, device=d)
        loops = torch.empty(i["n_loop"], dtype=torch.int32, device=d)
        self.ctx.check(load().pgcp_part_get_partition(self.ctx.h, self.h, _ptr(fl), _ptr(voff), _ptr(verts),
                                                      _ptr(loff), _ptr(loops)))
        return fl, voff, verts, loff, loops

    def local_param(self):
        self.ctx.check(load().pgcp_local_param(self.ctx.h, self.h))

    def csr(self):
        i = self.info()
        rp = torch.empty(i["n_copies"] + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(i["nnz"], dtype=torch.int32, device="cuda")
        val = torch.empty(i["nnz"], dtype=torch.float64, device="cuda")
        self.ctx.check(load().pgcp_part_get_csr(self.ctx.h, self.h, _ptr(rp), _ptr(col), _ptr(val)))
        return rp, col, val

    def coords(self, which: int):
        """0: DNCP (local frame), 1: welded / weld map, 2: final; complex128 [n_copies]."""
        i = self.info()
        out = torch.empty((i["n_copies"], 2), dtype=torch.float64, device="cuda")
        self.ctx.check(load().pgcp_part_get_coords(self.ctx.h, self.h, which, _ptr(out)))
        return torch.complex(out[:, 0], out[:, 1])

    def weld(self):
        self.ctx.check(load().pgcp_weld(self.ctx.h, self.h))

    def global_solve(self, out=None):
        dim = 3 if self.closed else 2
        if out is None:
            out = torch.empty((self.nv, dim), dtype=torch.float64, device="cuda")
        st = Stats()
        self.ctx.check(load().pgcp_global_solve(self.ctx.h, self.h, _ptr(out), 0, C.byref(st)))
        self.stats = st.as_dict()
        return out

    def metrics(self, U):
        check_coords(U, self.nv, self.closed, self.ctx.device)
        m = Distortion()
        self.ctx.check(load().pgcp_metrics(self.ctx.h, self.h, _ptr(U.contiguous()), C.byref(m)))
        return m.as_dict()

    def area_distortion(self, U):
        """pgcp_area_distortion: mean |d_area| (Section 6.2) of each mesh's planar map U."""
        check_coords(U, self.nv, self.closed, self.ctx.device)
        n = self.info()["n_mesh"]
        out = (C.c_double * n)()
        self.ctx.check(load().pgcp_area_distortion(self.ctx.h, self.h, _ptr(U.contiguous()), out))
        return list(out)

    def area_mobius(self, U, variant):
        """pgcp_area_mobius: the Mobius area step (Section 6.2) on U in place
        (a contiguous float64 CUDA tensor); one result dict per mesh."""
        check_coords(U, self.nv, self.closed, self.ctx.device, inplace=True)
        n = self.info()["n_mesh"]
        out = (AreaResult * n)()
        self.ctx.check(load().pgcp_area_mobius(self.ctx.h, self.h, _ptr(U), int(variant), out))
        return [r.as_dict() for r in out]

    def set_piece_mask(self, own):
        """pgcp_set_piece_mask: the pieces this part solves (sequence of K
        bools), or None for all."""
        if own is None:
            self.ctx.check(load().pgcp_set_piece_mask(self.ctx.h, self.h, None))
            return
        arr = np.ascontiguousarray(np.asarray(own, dtype=np.uint8))
        if arr.size != self.info()["K"]:
            raise ValueError("the mask needs one entry per piece")
        self.ctx.check(load().pgcp_set_piece_mask(self.ctx.h, self.h, arr.ctypes.data_as(C.c_void_p)))

    def get_boundary(self, which):
        """pgcp_part_get_boundary: [n_loop, 2] float64 CUDA tensor (0: local, 1: welded)."""
        out = torch.empty((self.info()["n_loop"], 2), dtype=torch.float64, device="cuda")
        self.ctx.check(load().pgcp_part_get_boundary(self.ctx.h, self.h, int(which), _ptr(out)))
        return out

    def set_boundary(self, which, B):
        """pgcp_part_set_boundary: import [n_loop, 2] boundary coordinates."""
        B = _dev(B, torch.float64).contiguous()
        if tuple(B.shape) != (self.info()["n_loop"], 2):
            raise ValueError("boundary coordinates must be [n_loop, 2]")
        self.ctx.check(load().pgcp_part_set_boundary(self.ctx.h, self.h, int(which), _ptr(B)))

    def fix_folds(self, U):
        """pgcp_fix_folds: the fold-over fix (Section 4.5, Algorithm 3) on the
        planar map U in place (contiguous float64 CUDA tensor [nv, 2]); returns
        the report dict."""
        check_coords(U, self.nv, self.closed, self.ctx.device, inplace=True)
        rep = FoldReport()
        self.ctx.check(load().pgcp_fix_folds(self.ctx.h, self.h, _ptr(U), C.byref(rep)))
        return rep.as_dict()

    def metrics_noalloc(self, U):
        """pgcp_metrics_noalloc: the same statistics with no device allocation,
        for callers that must not allocate (parts of at most
        METRICS_NOALLOC_MAX_FACES faces; calls must not overlap in time)."""
        check_coords(U, self.nv, self.closed, self.ctx.device)
        m = Distortion()
        self.ctx.check(load().pgcp_metrics_noalloc(self.ctx.h, self.h, _ptr(U.contiguous()), C.byref(m)))
        return m.as_dict()

    def free(self):
        if getattr(self, "h", None):
            load().pgcp_part_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Gnn:
    """The learned warm-start network (parameters live on the device)."""

    def __init__(self, ctx: Context, params=None, path: str | None = None):
        self.ctx = ctx
        h = C.c_void_p()
        if path is not None:
            ctx.check(load().pgcp_gnn_load(ctx.h, path.encode(), C.byref(h)))
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            if p.size != num_gnn_params():
                raise ValueError(f"expected {num_gnn_params()} parameters, got {p.size}")
            ctx.check(load().pgcp_gnn_create(ctx.h, p.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.h = h

    def params(self) -> np.ndarray:
        p = np.empty(num_gnn_params(), dtype=np.float32)
        self.ctx.check(load().pgcp_gnn_get_params(self.ctx.h, self.h, p.ctypes.data_as(C.c_void_p)))
        return p

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self.ctx.check(load().pgcp_gnn_set_params(self.ctx.h, self.h, p.ctypes.data_as(C.c_void_p)))

    def grad(self, part):
        g = np.empty(num_gnn_params(), dtype=np.float32)
        l = C.c_double()
        self.ctx.check(load().pgcp_gnn_grad(self.ctx.h, self.h, part.h, g.ctypes.data_as(C.c_void_p), C.byref(l)))
        return g, l.value

    def train_step(self, part, lr: float) -> float:
        l = C.c_double()
        self.ctx.check(load().pgcp_gnn_train_step(self.ctx.h, self.h, part.h, C.c_float(lr), C.byref(l)))
        return l.value

    def predict(self, part):
        rows = part.info()["n_copies"]
        x = torch.empty((rows, 2), dtype=torch.float64, device="cuda")
        self.ctx.check(load().pgcp_gnn_predict(self.ctx.h, self.h, part.h, _ptr(x)))
        return x

    def free(self):
        if getattr(self, "h", None):
            load().pgcp_gnn_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def num_gnn_params() -> int:
    return int(load().pgcp_gnn_num_params())


def gnn_inputs(part, targets: bool = True):
    """(features [rows, 16], targets [rows, 2] or None, sigma [K]) as CUDA tensors."""
    i = part.info()
    feat = torch.empty((i["n_copies"], 16), dtype=torch.float32, device="cuda")
    tgt = torch.empty((i["n_copies"], 2), dtype=torch.float32, device="cuda") if targets else None
    sig = torch.empty(i["K"], dtype=torch.float32, device="cuda")
    part.ctx.check(load().pgcp_gnn_inputs(part.ctx.h, part.h, _ptr(feat), _ptr(tgt), _ptr(sig)))
    return feat, tgt, sig
