"""Python binding of libgf2x_gb300 (include/gf2x_gb300.h).

Argument marshalling only: every step of the product runs in the CUDA kernels
of the shared library; nothing here computes.  The functions carry the C ABI's
names and arguments.  Device buffers are passed as PyTorch CUDA tensors (any
integer dtype; their bytes are the little-endian uint64 words), host buffers
as numpy arrays, streams as torch.cuda.Stream (or None for the legacy default
stream).  A non-zero status raises GF2XError.

The library must be built first (paper_1708_09746_gb300.build); loading fails
loudly if it is missing -- there is no fallback implementation.
"""
import ctypes
import os

__all__ = [
    "GF2XError", "load", "gf2x_strerror", "gf2x_out_words", "gf2x_fft_points", "gf2x_chunking",
    "gf2x_mul", "gf2x_mul_async", "gf2x_mul_host", "gf2x_plan_create",
    "gf2x_plan_workspace_bytes", "gf2x_plan_execute", "gf2x_plan_destroy",
    "gf2x_mul_batched", "gf2x_stage_basis_cvt64", "gf2x_stage_basis_cvt128",
    "gf2x_stage_chrepr", "gf2x_stage_fft", "gf2x_stage_pointmul",
    "gf2x_stage_ichrepr_combine", "gf2x_shutdown", "gf2x_profile_enable",
    "gf2x_profile_reset", "gf2x_profile_read", "gf2x_profile_stage_name", "gf2x_mul_noalloc",
    "gf2x_batch_create", "gf2x_batch_workspace_bytes", "gf2x_batch_execute", "gf2x_batch_destroy",
    "gf2x_server_create", "gf2x_server_submit", "gf2x_server_wait", "gf2x_server_stats",
    "gf2x_server_reset_stats", "gf2x_server_destroy", "gf2x_probe_pipes", "LIB_PATH",
    "gf2x_stream_status", "gf2x_batch_status", "gf2x_debug_set_wait_spins",
    "gf2x_tower256_fft_points", "gf2x_mul_tower256", "gf2x_mul_tower256_async",
    "gf2x_stage_chrepr256", "gf2x_stage_pointmul256", "gf2x_stage_ichrepr256_combine",
    "gf2x_mul_simple", "gf2x_mul_simple_async", "gf2x_stage_fft_simple", "gf2x_stage_gfmul_simple",
    "gf2x_frobenius_points", "gf2x_mul_frobenius", "gf2x_mul_frobenius_async",
    "gf2x_stage_bit_basis_cvt", "gf2x_stage_frobenius_encode", "gf2x_stage_fft_frobenius",
    "gf2x_product_path", "gf2x_batch_tune",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgf2x_gb300.so")

GF2X_OK, GF2X_EINVAL, GF2X_ENOMEM, GF2X_ECUDA, GF2X_ETIMEOUT, GF2X_EBUSY = 0, -1, -2, -3, -4, -5


class GF2XError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, gf2x_strerror(status), status))


_lib = None
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p
_int = ctypes.c_int

class gf2x_tune_t(ctypes.Structure):
    """Plan parameters of one transform shape (include/gf2x_gb300.h)."""
    _fields_ = [("fft_depth", ctypes.c_int), ("fft_buffers", ctypes.c_int),
                ("bcvt_tile_log", ctypes.c_int), ("bcvt_threads", ctypes.c_int),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {"fft_depth": self.fft_depth, "fft_buffers": self.fft_buffers,
                "bcvt_tile_log": self.bcvt_tile_log, "bcvt_threads": self.bcvt_threads,
                "ms": self.ms}


_SIGS = {
    "gf2x_strerror": (ctypes.c_char_p, [_int]),
    "gf2x_out_words": (_u64, [_u64, _u64]),
    "gf2x_fft_points": (_u64, [_u64, _u64]),
    "gf2x_chunking": (_int, [_u64, _u64, ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "gf2x_mul": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_mul_async": (_int, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "gf2x_mul_host": (_int, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "gf2x_plan_create": (_int, [_u64, _u64, ctypes.POINTER(_vp)]),
    "gf2x_plan_workspace_bytes": (_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "gf2x_plan_execute": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "gf2x_plan_destroy": (_int, [_vp]),
    "gf2x_mul_batched": (_int, [_int, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gf2x_stage_basis_cvt64": (_int, [_vp, _int, _int, _vp]),
    "gf2x_stage_basis_cvt128": (_int, [_vp, _int, _int, _vp]),
    "gf2x_stage_chrepr": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_stage_fft": (_int, [_vp, _int, _int, _int, _vp]),
    "gf2x_stage_pointmul": (_int, [_vp, _vp, _vp, _u64, _vp]),
    "gf2x_stage_ichrepr_combine": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_shutdown": (_int, []),
    "gf2x_profile_enable": (_int, [_int]),
    "gf2x_profile_reset": (_int, []),
    "gf2x_profile_read": (_int, [_int, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "gf2x_profile_stage_name": (ctypes.c_char_p, [_int]),
    "gf2x_probe_pipes": (_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "gf2x_mul_noalloc": (_int, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "gf2x_batch_create": (_int, [_int, _vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "gf2x_batch_workspace_bytes": (_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "gf2x_batch_execute": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "gf2x_batch_destroy": (_int, [_vp]),
    "gf2x_server_create": (_int, [ctypes.c_size_t, _int, _int, ctypes.POINTER(_vp)]),
    "gf2x_server_submit": (_int, [_vp, _vp, _u64, _vp, _u64, _vp, ctypes.POINTER(_u64)]),
    "gf2x_server_wait": (_int, [_vp, _u64, _u64]),
    "gf2x_server_stats": (_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_u64)]),
    "gf2x_server_reset_stats": (_int, [_vp]),
    "gf2x_server_destroy": (_int, [_vp]),
    "gf2x_autotune": (_int, [_u64, _u64, _int, ctypes.POINTER(gf2x_tune_t)]),
    "gf2x_tune_get": (_int, [_u64, _u64, ctypes.POINTER(gf2x_tune_t)]),
    "gf2x_tune_set": (_int, [_u64, _u64, ctypes.POINTER(gf2x_tune_t)]),
    "gf2x_tune_save": (_int, [ctypes.c_char_p]),
    "gf2x_tune_load": (_int, [ctypes.c_char_p]),
    "gf2x_stream_status": (_int, [_vp]),
    "gf2x_batch_status": (_int, [_vp]),
    "gf2x_debug_set_wait_spins": (_int, [ctypes.c_int64]),
    "gf2x_tower256_fft_points": (_u64, [_u64, _u64]),
    "gf2x_mul_tower256": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_mul_tower256_async": (_int, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "gf2x_stage_chrepr256": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_stage_pointmul256": (_int, [_vp, _vp, _u64, _vp]),
    "gf2x_stage_ichrepr256_combine": (_int, [_vp, _u64, _vp, _u64, _u64, _vp]),
    "gf2x_mul_simple": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_mul_simple_async": (_int, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "gf2x_stage_fft_simple": (_int, [_vp, _int, _int, _int, _vp]),
    "gf2x_stage_gfmul_simple": (_int, [_vp, _vp, _u64, _vp]),
    "gf2x_frobenius_points": (_int, [_u64, _u64]),
    "gf2x_mul_frobenius": (_int, [_vp, _u64, _vp, _u64, _vp]),
    "gf2x_mul_frobenius_async": (_int, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "gf2x_stage_bit_basis_cvt": (_int, [_vp, _int, _int, _vp]),
    "gf2x_stage_frobenius_encode": (_int, [_vp, _int, _int, _vp, _int, _vp]),
    "gf2x_stage_fft_frobenius": (_int, [_vp, _int, _int, _vp]),
    "gf2x_product_path": (_int, [_u64, _u64, ctypes.POINTER(_int), ctypes.POINTER(_u64),
                                 ctypes.POINTER(_u64)]),
    "gf2x_batch_tune": (_int, [_vp, _int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]),
}


def load():
    """Load the shared library (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libgf2x_gb300.so is not built (run "
                          "`python -m paper_1708_09746_gb300.build`): " + LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Raw address of a torch tensor / numpy array / int (None -> 0)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, where):
    if rc != GF2X_OK:
        raise GF2XError(rc, where)


def gf2x_strerror(status):
    return load().gf2x_strerror(int(status)).decode()


def gf2x_out_words(na_bits, nb_bits):
    return int(load().gf2x_out_words(na_bits, nb_bits))


def gf2x_fft_points(na_bits, nb_bits):
    return int(load().gf2x_fft_points(na_bits, nb_bits))


def gf2x_chunking(na_bits, nb_bits):
    """(chunk words, chunks, points per chunk transform) of the one-shot calls'
    chunked product; (0, 0, 0) when the product is one transform."""
    L, C, N = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().gf2x_chunking(na_bits, nb_bits, ctypes.byref(L), ctypes.byref(C), ctypes.byref(N)),
           "gf2x_chunking")
    return int(L.value), int(C.value), int(N.value)


def gf2x_mul(a, na_bits, b, nb_bits, out):
    _check(load().gf2x_mul(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out)), "gf2x_mul")


def gf2x_mul_async(a, na_bits, b, nb_bits, out, stream=None):
    _check(load().gf2x_mul_async(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out), _stream(stream)),
           "gf2x_mul_async")


def gf2x_mul_host(a_host, na_bits, b_host, nb_bits, out_host, stream=None):
    _check(load().gf2x_mul_host(_ptr(a_host), na_bits, _ptr(b_host), nb_bits, _ptr(out_host),
                                _stream(stream)), "gf2x_mul_host")


def gf2x_mul_noalloc(a, na_bits, b, nb_bits, out, stream=None):
    """gf2x_mul for callers that cannot allocate device memory: the scratch
    is a static device array of the library (see include/gf2x_gb300.h)."""
    _check(load().gf2x_mul_noalloc(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out),
                                   _stream(stream)), "gf2x_mul_noalloc")


def gf2x_autotune(na_bits, nb_bits, reps=3):
    """Times candidate plan parameters for this product shape on the current
    device, stores the fastest for the shape and returns them as a dict."""
    t = gf2x_tune_t()
    _check(load().gf2x_autotune(na_bits, nb_bits, int(reps), ctypes.byref(t)), "gf2x_autotune")
    return t.as_dict()


def gf2x_tune_get(na_bits, nb_bits):
    t = gf2x_tune_t()
    _check(load().gf2x_tune_get(na_bits, nb_bits, ctypes.byref(t)), "gf2x_tune_get")
    return t.as_dict()


def gf2x_tune_set(na_bits, nb_bits, fft_depth, fft_buffers, bcvt_tile_log, bcvt_threads, ms=-1.0):
    t = gf2x_tune_t(int(fft_depth), int(fft_buffers), int(bcvt_tile_log), int(bcvt_threads),
                    float(ms))
    _check(load().gf2x_tune_set(na_bits, nb_bits, ctypes.byref(t)), "gf2x_tune_set")


def gf2x_tune_save(path):
    _check(load().gf2x_tune_save(os.fsencode(path)), "gf2x_tune_save")


def gf2x_tune_load(path):
    _check(load().gf2x_tune_load(os.fsencode(path)), "gf2x_tune_load")


def gf2x_plan_create(na_bits, nb_bits):
    p = _vp()
    _check(load().gf2x_plan_create(na_bits, nb_bits, ctypes.byref(p)), "gf2x_plan_create")
    return p.value


def gf2x_plan_workspace_bytes(plan):
    n = ctypes.c_size_t()
    _check(load().gf2x_plan_workspace_bytes(plan, ctypes.byref(n)), "gf2x_plan_workspace_bytes")
    return int(n.value)


def gf2x_plan_execute(plan, a, b, out, workspace=None, stream=None):
    _check(load().gf2x_plan_execute(plan, _ptr(a), _ptr(b), _ptr(out), _ptr(workspace),
                                    _stream(stream)), "gf2x_plan_execute")


def gf2x_plan_destroy(plan):
    _check(load().gf2x_plan_destroy(plan), "gf2x_plan_destroy")


def gf2x_mul_batched(a_list, na_bits, b_list, nb_bits, out_list, stream=None):
    n = len(a_list)
    P = ctypes.c_void_p * n
    U = ctypes.c_uint64 * n
    pa, pb, po = P(*[_ptr(x) for x in a_list]), P(*[_ptr(x) for x in b_list]), \
        P(*[_ptr(x) for x in out_list])
    na, nb = U(*[int(x) for x in na_bits]), U(*[int(x) for x in nb_bits])
    _check(load().gf2x_mul_batched(n, ctypes.cast(pa, _vp), ctypes.cast(na, _vp),
                                   ctypes.cast(pb, _vp), ctypes.cast(nb, _vp),
                                   ctypes.cast(po, _vp), _stream(stream)), "gf2x_mul_batched")


def gf2x_stage_basis_cvt64(f, log_n, inverse=0, stream=None):
    _check(load().gf2x_stage_basis_cvt64(_ptr(f), log_n, inverse, _stream(stream)),
           "gf2x_stage_basis_cvt64")


def gf2x_stage_basis_cvt128(f, log_n, inverse=0, stream=None):
    _check(load().gf2x_stage_basis_cvt128(_ptr(f), log_n, inverse, _stream(stream)),
           "gf2x_stage_basis_cvt128")


def gf2x_stage_chrepr(g, p, F, n, stream=None):
    _check(load().gf2x_stage_chrepr(_ptr(g), p, _ptr(F), n, _stream(stream)), "gf2x_stage_chrepr")


def gf2x_stage_fft(F, log_n, log_p, inverse=0, stream=None):
    _check(load().gf2x_stage_fft(_ptr(F), log_n, log_p, inverse, _stream(stream)),
           "gf2x_stage_fft")


def gf2x_stage_pointmul(A, B, C, n, stream=None):
    _check(load().gf2x_stage_pointmul(_ptr(A), _ptr(B), _ptr(C), n, _stream(stream)),
           "gf2x_stage_pointmul")


def gf2x_stage_ichrepr_combine(F, n, out, total_bits, stream=None):
    _check(load().gf2x_stage_ichrepr_combine(_ptr(F), n, _ptr(out), total_bits, _stream(stream)),
           "gf2x_stage_ichrepr_combine")


def gf2x_shutdown():
    _check(load().gf2x_shutdown(), "gf2x_shutdown")


def gf2x_profile_enable(on=1):
    _check(load().gf2x_profile_enable(int(on)), "gf2x_profile_enable")


def gf2x_profile_reset():
    _check(load().gf2x_profile_reset(), "gf2x_profile_reset")


def gf2x_profile_read(stage):
    """(ms, launches, calls) summed for stage index `stage`."""
    ms = ctypes.c_double()
    la = ctypes.c_uint64()
    ca = ctypes.c_uint64()
    _check(load().gf2x_profile_read(int(stage), ctypes.byref(ms), ctypes.byref(la),
                                    ctypes.byref(ca)), "gf2x_profile_read")
    return float(ms.value), int(la.value), int(ca.value)


def gf2x_profile_stage_name(stage):
    return load().gf2x_profile_stage_name(int(stage)).decode()


def gf2x_probe_pipes():
    """Issue rates (warp instructions per SM clock) of shfl.sync.idx, lop3 and
    conflict-free shared-memory loads on the current device, and its SM count."""
    sh, xo, ld = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int()
    _check(load().gf2x_probe_pipes(ctypes.byref(sh), ctypes.byref(xo), ctypes.byref(ld),
                                   ctypes.byref(n)), "gf2x_probe_pipes")
    return {"shfl_per_clk_sm": sh.value, "xor_per_clk_sm": xo.value,
            "lds_per_clk_sm": ld.value, "sms": n.value}


def profile_all():
    """{stage name: (ms, launches, calls)} for every stage."""
    out = {}
    i = 0
    while True:
        name = gf2x_profile_stage_name(i)
        if not name:
            return out
        out[name] = gf2x_profile_read(i)
        i += 1


def _u64_array(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_uint64 * len(vals))(*vals)


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])


def gf2x_batch_create(na_bits, nb_bits, mem_budget_bytes=0):
    """Reusable batch for these per-product sizes; returns an opaque handle."""
    if len(na_bits) != len(nb_bits):
        raise ValueError("size lists differ in length")
    h = _vp()
    na, nb = _u64_array(na_bits), _u64_array(nb_bits)
    _check(load().gf2x_batch_create(len(na), ctypes.cast(na, _vp), ctypes.cast(nb, _vp),
                                    int(mem_budget_bytes), ctypes.byref(h)), "gf2x_batch_create")
    return h.value


def gf2x_batch_workspace_bytes(batch):
    n = ctypes.c_size_t()
    _check(load().gf2x_batch_workspace_bytes(batch, ctypes.byref(n)), "gf2x_batch_workspace_bytes")
    return int(n.value)


def gf2x_batch_execute(batch, a_list, b_list, out_list, stream=None):
    pa, pb, po = _ptr_array(a_list), _ptr_array(b_list), _ptr_array(out_list)
    _check(load().gf2x_batch_execute(batch, ctypes.cast(pa, _vp), ctypes.cast(pb, _vp),
                                     ctypes.cast(po, _vp), _stream(stream)), "gf2x_batch_execute")


def gf2x_batch_destroy(batch):
    _check(load().gf2x_batch_destroy(batch), "gf2x_batch_destroy")


def gf2x_server_create(mem_budget_bytes, max_slots, max_batch=64):
    h = _vp()
    _check(load().gf2x_server_create(int(mem_budget_bytes), int(max_slots), int(max_batch),
                                     ctypes.byref(h)), "gf2x_server_create")
    return h.value


def gf2x_server_submit(server, a, na_bits, b, nb_bits, out):
    t = ctypes.c_uint64()
    _check(load().gf2x_server_submit(server, _ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out),
                                     ctypes.byref(t)), "gf2x_server_submit")
    return int(t.value)


def gf2x_server_wait(server, ticket, timeout_us):
    """Status of the ticket (0), raises on error; GF2X_ETIMEOUT raises too."""
    _check(load().gf2x_server_wait(server, int(ticket), int(timeout_us)), "gf2x_server_wait")


def gf2x_server_stats(server):
    """(p50_ms, p99_ms, throughput_per_s, completed)."""
    p50, p99, thr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_uint64()
    _check(load().gf2x_server_stats(server, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(thr),
                                    ctypes.byref(n)), "gf2x_server_stats")
    return float(p50.value), float(p99.value), float(thr.value), int(n.value)


def gf2x_server_reset_stats(server):
    _check(load().gf2x_server_reset_stats(server), "gf2x_server_reset_stats")


def gf2x_server_destroy(server):
    _check(load().gf2x_server_destroy(server), "gf2x_server_destroy")


def gf2x_stream_status(stream=None):
    """Waits for `stream`; raises GF2XError(GF2X_ETIMEOUT) if a bounded device
    wait of an asynchronous call on it ran out since the last check."""
    _check(load().gf2x_stream_status(_stream(stream)), "gf2x_stream_status")


def gf2x_batch_status(batch):
    """Waits for the batch's last execution; raises GF2XError(GF2X_ETIMEOUT)
    if a bounded device wait in it ran out."""
    _check(load().gf2x_batch_status(batch), "gf2x_batch_status")


def gf2x_debug_set_wait_spins(spins):
    """Bound of the kernels' device waits for tests of the timeout path
    (0: give up at once; negative: the default)."""
    _check(load().gf2x_debug_set_wait_spins(int(spins)), "gf2x_debug_set_wait_spins")


def gf2x_tower256_fft_points(na_bits, nb_bits):
    return int(load().gf2x_tower256_fft_points(na_bits, nb_bits))


def gf2x_mul_tower256(a, na_bits, b, nb_bits, out):
    """c = a * b by the F~_{2^256} (w = 128) form, synchronous."""
    _check(load().gf2x_mul_tower256(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out)),
           "gf2x_mul_tower256")


def gf2x_mul_tower256_async(a, na_bits, b, nb_bits, out, stream=None):
    _check(load().gf2x_mul_tower256_async(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out),
                                          _stream(stream)), "gf2x_mul_tower256_async")


def gf2x_stage_chrepr256(blocks, P, F, N2, stream=None):
    _check(load().gf2x_stage_chrepr256(_ptr(blocks), P, _ptr(F), N2, _stream(stream)),
           "gf2x_stage_chrepr256")


def gf2x_stage_pointmul256(A, B, N2, stream=None):
    _check(load().gf2x_stage_pointmul256(_ptr(A), _ptr(B), N2, _stream(stream)),
           "gf2x_stage_pointmul256")


def gf2x_stage_ichrepr256_combine(F, N2, out, out_words, total_bits, stream=None):
    _check(load().gf2x_stage_ichrepr256_combine(_ptr(F), N2, _ptr(out), out_words, total_bits,
                                                _stream(stream)), "gf2x_stage_ichrepr256_combine")


def gf2x_mul_simple(a, na_bits, b, nb_bits, out):
    """c = a * b by the simple polynomial-basis form (Alg. 4), synchronous."""
    _check(load().gf2x_mul_simple(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out)), "gf2x_mul_simple")


def gf2x_mul_simple_async(a, na_bits, b, nb_bits, out, stream=None):
    _check(load().gf2x_mul_simple_async(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out),
                                        _stream(stream)), "gf2x_mul_simple_async")


def gf2x_stage_fft_simple(F, log_n, layers, inverse, stream=None):
    _check(load().gf2x_stage_fft_simple(_ptr(F), int(log_n), int(layers), int(inverse),
                                        _stream(stream)), "gf2x_stage_fft_simple")


def gf2x_stage_gfmul_simple(A, B, n, stream=None):
    _check(load().gf2x_stage_gfmul_simple(_ptr(A), _ptr(B), n, _stream(stream)),
           "gf2x_stage_gfmul_simple")


def gf2x_frobenius_points(na_bits, nb_bits):
    return int(load().gf2x_frobenius_points(na_bits, nb_bits))


def gf2x_mul_frobenius(a, na_bits, b, nb_bits, out):
    """c = a * b by the Frobenius-partition form (Appendix C), synchronous."""
    _check(load().gf2x_mul_frobenius(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out)),
           "gf2x_mul_frobenius")


def gf2x_mul_frobenius_async(a, na_bits, b, nb_bits, out, stream=None):
    _check(load().gf2x_mul_frobenius_async(_ptr(a), na_bits, _ptr(b), nb_bits, _ptr(out),
                                           _stream(stream)), "gf2x_mul_frobenius_async")


def gf2x_stage_bit_basis_cvt(f, log_bits, inverse, stream=None):
    _check(load().gf2x_stage_bit_basis_cvt(_ptr(f), int(log_bits), int(inverse), _stream(stream)),
           "gf2x_stage_bit_basis_cvt")


def gf2x_stage_frobenius_encode(g, log_bits, m, E, decode, stream=None):
    _check(load().gf2x_stage_frobenius_encode(_ptr(g), int(log_bits), int(m), _ptr(E), int(decode),
                                              _stream(stream)), "gf2x_stage_frobenius_encode")


def gf2x_stage_fft_frobenius(F, m, inverse, stream=None):
    _check(load().gf2x_stage_fft_frobenius(_ptr(F), int(m), int(inverse), _stream(stream)),
           "gf2x_stage_fft_frobenius")


def gf2x_product_path(na_bits, nb_bits):
    """(path, main_a_words, main_b_words) of the one-shot calls: path 0 one
    transform, 1 chunks, 2 direct (short operand), 3 tail split."""
    p, A, B = _int(), _u64(), _u64()
    _check(load().gf2x_product_path(na_bits, nb_bits, ctypes.byref(p), ctypes.byref(A), ctypes.byref(B)),
           "gf2x_product_path")
    return int(p.value), int(A.value), int(B.value)


def gf2x_batch_tune(batch, reps=2):
    """Tunes each shape group of the batch on its own grouped launch (after one
    execution); returns (ms_before, ms_after) summed over the groups."""
    b, a = ctypes.c_double(), ctypes.c_double()
    _check(load().gf2x_batch_tune(batch, int(reps), ctypes.byref(b), ctypes.byref(a)), "gf2x_batch_tune")
    return float(b.value), float(a.value)
