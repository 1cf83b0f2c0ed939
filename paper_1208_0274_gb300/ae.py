"""Python binding of libae (include/ae.h): argument marshalling only.

Every function here has the name and meaning of the C entry point it wraps;
all compute happens in the library's CUDA kernels.  The library is loaded
from this package directory; if it is missing the import of this module
fails with an error naming the build command (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libae.so")

AE_OK, AE_EINVAL, AE_ENOMEM, AE_EOVERFLOW, AE_ETIMEOUT, AE_ECUDA, AE_EUNSUPPORTED, AE_EIO = range(8)
AE_DNA, AE_PROTEIN = 0, 1
ALPHABETS = {AE_DNA: b"ACGT", AE_PROTEIN: b"ARNDCQEGHILKMFPSTWYV"}

HIT_DTYPE = np.dtype([("text_end", "<i8"), ("query_end", "<i4"), ("score", "<i4")])


class AEError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class ae_scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("matrix", ctypes.c_void_p), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32)]


class ae_query(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_void_p), ("len", ctypes.c_int64)]


class ae_options(ctypes.Structure):
    _fields_ = [("qprefix_seed", ctypes.c_int32), ("leaf_segment", ctypes.c_int32),
                ("item_columns", ctypes.c_int64), ("batch_columns", ctypes.c_int64),
                ("leaf_capacity", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("leaf_delay", ctypes.c_int32), ("int16_limit", ctypes.c_int32),
                ("hint_hits", ctypes.c_void_p), ("tier_stats", ctypes.c_int32),
                ("workspace_limit", ctypes.c_int64), ("general_rows", ctypes.c_int32),
                ("qprefix_domination", ctypes.c_int32), ("row_layout", ctypes.c_int32),
                ("fork_parts", ctypes.c_int32), ("fork_part", ctypes.c_int32),
                ("leaf_wide_rows", ctypes.c_int32)]


class ae_stats(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_int64), ("leaf_rows", ctypes.c_int64),
                ("entries", ctypes.c_int64), ("entries_tier", ctypes.c_int64 * 3),
                ("injections", ctypes.c_int64), ("raw_hits", ctypes.c_int64),
                ("hits", ctypes.c_int64), ("entries_leaf", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("levels_int16", ctypes.c_int32), ("seed_depth", ctypes.c_int32), ("ms_trie", ctypes.c_double),
                ("ms_leaf", ctypes.c_double), ("ms_reduce", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_k_expand", ctypes.c_double),
                ("ms_k_leaf", ctypes.c_double), ("ms_k_sort", ctypes.c_double),
                ("ms_k_other", ctypes.c_double), ("ms_k_rows", ctypes.c_double),
                ("leaf_max_steps", ctypes.c_int64),
                ("leaf_max_width", ctypes.c_int64), ("ws_bytes", ctypes.c_int64),
                ("leaf_sweeps", ctypes.c_int64), ("leaf_raw_hits", ctypes.c_int64),
                ("triples", ctypes.c_int64), ("batch_splits", ctypes.c_int64),
                ("dominated", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("pruned_nonpos", ctypes.c_int64), ("pruned_reach", ctypes.c_int64),
                ("reused", ctypes.c_int64), ("reroutes", ctypes.c_int64),
                ("leaf_wide_walks", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIBPATH)
    V, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "ae_options_default": (None, [V]),
        "ae_strerror": (ctypes.c_char_p, [I32]),
        "ae_index_build": (I32, [V, I64, I32, V]),
        "ae_index_build_collection": (I32, [V, I64, V, I32, I32, V]),
        "ae_index_save": (I32, [V, ctypes.c_char_p]),
        "ae_index_load": (I32, [ctypes.c_char_p, V]),
        "ae_index_free": (None, [V]),
        "ae_index_info": (I32, [V, V, V, V]),
        "ae_search": (I32, [V, V, I32, V, V, V, V, V, V]),
        "ae_hits_free": (None, [V]),
        "ae_search_device": (I32, [V, V, V, I32, V, V, V, V, I64, V, V]),
        "ae_search_device_static": (I32, [V, V, V, I32, V, V, V, V, I64, V, V]),
        "ae_workspace_info": (I32, [V, V, V, V]),
        "ae_hits_merge": (I32, [V, V, I64, I32, I64, I64, V, V, V, V]),
        "ae_mlp_create": (I32, [ctypes.c_uint64, V]),
        "ae_mlp_free": (None, [V]),
        "ae_mlp_set_params": (I32, [V, V]),
        "ae_mlp_get_params": (I32, [V, V]),
        "ae_mlp_set_norm": (I32, [V, V, V, V, V]),
        "ae_mlp_features": (I32, [V, V, V, I32, V, V]),
        "ae_mlp_forward": (I32, [V, V, I32, V, V]),
        "ae_mlp_loss_grad": (I32, [V, V, V, I32, V, V, V]),
        "ae_mlp_train": (I32, [V, V, V, I32, I32, I32, ctypes.c_float, ctypes.c_float, ctypes.c_uint64, V, V]),
        "ae_workspace_release": (I32, [V, V]),
        "ae_last_stats": (I32, [V]),
        "ae_suffix_array": (I32, [V, I64, I32, V]),
        "ae_suffix_array_device": (I32, [V, I64, I32, I32, V, V]),
        "ae_plan": (I32, [I64, I32, V, I32, V, V, V]),
        "ae_int_peak": (I32, [I32, I32, I32, I32, V, V, V, V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def strerror(status):
    return lib.ae_strerror(int(status)).decode()


def _check(st, where):
    if st != AE_OK:
        raise AEError(st, where)


def _u8(seq):
    if isinstance(seq, str):
        seq = seq.encode()
    if isinstance(seq, (bytes, bytearray)):
        return np.frombuffer(bytes(seq), dtype=np.uint8)
    return np.ascontiguousarray(np.asarray(seq, dtype=np.uint8))


def make_scoring(scheme, alphabet=AE_DNA):
    """ae_scoring from any object with match / mismatch / gap_open /
    gap_extend (/ matrix) attributes, or a dict with those keys. Returns the
    struct and the matrix buffer it points to (keep both alive)."""
    get = (lambda k, d=None: scheme.get(k, d)) if isinstance(scheme, dict) else \
        (lambda k, d=None: getattr(scheme, k, d))
    s = ae_scoring()
    s.match = int(get("match", 1))
    s.mismatch = int(get("mismatch", -3))
    s.gap_open = int(get("gap_open", -5))
    s.gap_extend = int(get("gap_extend", -2))
    mat = get("matrix", None)
    buf = None
    if mat is not None:
        buf = np.ascontiguousarray(np.asarray(mat, dtype=np.int8))
        s.matrix = buf.ctypes.data
    else:
        s.matrix = None
    return s, buf


def ae_options_default():
    o = ae_options()
    lib.ae_options_default(ctypes.byref(o))
    return o


def make_options(hint_hits=None, **kw):
    """ae_options with the given fields set.  hint_hits: per-query expected
    sweep hit records (kept alive on the returned object)."""
    o = ae_options_default()
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, int(v))
    if hint_hits is not None:
        h = np.ascontiguousarray(np.asarray(hint_hits, dtype=np.int64))
        o._hint_ref = h
        o.hint_hits = h.ctypes.data
    return o


class Index:
    """Owns one ae_index*; freed with ae_index_free."""

    def __init__(self, handle, alphabet):
        self._h = ctypes.c_void_p(handle)
        self.alphabet = alphabet

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h and self._h.value:
            lib.ae_index_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ae_index_build(text, alphabet=AE_DNA):
    t = _u8(text)
    out = ctypes.c_void_p(0)
    _check(lib.ae_index_build(t.ctypes.data, t.size, int(alphabet), ctypes.byref(out)), "ae_index_build")
    return Index(out.value, alphabet)


def ae_index_build_collection(sequences, alphabet=AE_DNA):
    """Index of a collection: `sequences` is a list of sequences (ASCII), joined
    back to back; results report positions in that concatenation, and no
    alignment spans two sequences."""
    seqs = [_u8(q) for q in sequences]
    t = np.concatenate(seqs) if seqs else np.zeros(0, np.uint8)
    starts = np.ascontiguousarray(np.concatenate([[0], np.cumsum([q.size for q in seqs])[:-1]]).astype(np.int64))
    out = ctypes.c_void_p(0)
    _check(lib.ae_index_build_collection(t.ctypes.data, t.size, starts.ctypes.data, len(seqs), int(alphabet),
                                         ctypes.byref(out)), "ae_index_build_collection")
    return Index(out.value, alphabet)


def ae_index_save(index, path):
    _check(lib.ae_index_save(index.handle, str(path).encode()), "ae_index_save")


def ae_index_load(path):
    out = ctypes.c_void_p(0)
    _check(lib.ae_index_load(str(path).encode(), ctypes.byref(out)), "ae_index_load")
    n, a, b = ae_index_info_raw(out)
    return Index(out.value, a)


def ae_index_info_raw(handle):
    n = ctypes.c_int64()
    a = ctypes.c_int32()
    b = ctypes.c_int64()
    _check(lib.ae_index_info(handle, ctypes.byref(n), ctypes.byref(a), ctypes.byref(b)), "ae_index_info")
    return n.value, a.value, b.value


def ae_index_info(index):
    n, a, b = ae_index_info_raw(index.handle)
    return {"n": n, "alphabet": a, "device_bytes": b}


def _thresholds(H, nq):
    h = np.full(nq, H, dtype=np.int32) if np.isscalar(H) else np.ascontiguousarray(np.asarray(H, dtype=np.int32))
    if h.size != nq:
        raise ValueError("one threshold per query")
    return h


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def ae_search(index, queries, scheme, H, options=None, stream=None):
    """Host queries in, host results out. Returns (hits, counts): hits is a
    structured array (text_end, query_end, score) grouped by query and sorted
    by (text_end, query_end); counts[k] is query k's number of results."""
    qs = [_u8(q) for q in queries]
    nq = len(qs)
    arr = (ae_query * max(nq, 1))()
    for k, q in enumerate(qs):
        arr[k].seq = q.ctypes.data if q.size else None
        arr[k].len = q.size
    h = _thresholds(H, nq)
    sc, _mat = make_scoring(scheme, index.alphabet)
    out = ctypes.c_void_p(0)
    counts = np.zeros(max(nq, 1), dtype=np.int64)
    st = lib.ae_search(index.handle, ctypes.cast(arr, ctypes.c_void_p), nq, ctypes.byref(sc),
                       h.ctypes.data, ctypes.byref(options) if options is not None else None,
                       ctypes.byref(out), counts.ctypes.data, _stream_handle(stream))
    _check(st, "ae_search")
    total = int(counts[:nq].sum())
    if not total:
        lib.ae_hits_free(out)
        return np.empty(0, dtype=HIT_DTYPE), counts[:nq].copy()
    # the array is a view of the library's buffer, which is freed when the last
    # array over it goes away (no second copy of the results)
    buf = (ctypes.c_uint8 * (total * HIT_DTYPE.itemsize)).from_address(out.value)
    weakref.finalize(buf, lib.ae_hits_free, ctypes.c_void_p(out.value))
    return np.frombuffer(buf, dtype=HIT_DTYPE, count=total), counts[:nq].copy()


def ae_search_device(index, d_seq_ptr, offsets, scheme, H, d_hits_ptr, capacity, options=None, stream=None):
    """Device-resident queries (d_seq_ptr: device address of the ASCII letters
    back to back; offsets: host int64 nq+1) and results (d_hits_ptr: device
    buffer of `capacity` 16-byte hits). Returns (status, counts); status is
    AE_OK or AE_EOVERFLOW (counts then hold the sizes needed)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nq = off.size - 1
    h = _thresholds(H, nq)
    sc, _mat = make_scoring(scheme, index.alphabet)
    counts = np.zeros(max(nq, 1), dtype=np.int64)
    st = lib.ae_search_device(index.handle, ctypes.c_void_p(int(d_seq_ptr)), off.ctypes.data, nq,
                              ctypes.byref(sc), h.ctypes.data,
                              ctypes.byref(options) if options is not None else None,
                              ctypes.c_void_p(int(d_hits_ptr)) if d_hits_ptr else None, int(capacity),
                              counts.ctypes.data, _stream_handle(stream))
    if st not in (AE_OK, AE_EOVERFLOW):
        _check(st, "ae_search_device")
    return st, counts[:nq].copy()


def ae_search_device_static(index, d_seq_ptr, offsets, scheme, H, d_hits_ptr, capacity, options=None,
                            stream=None):
    """ae_search_device without any device allocation: working memory comes
    from a fixed array inside the library (limits in include/ae.h). Returns
    (status, counts) like ae_search_device; AE_EUNSUPPORTED when the problem
    exceeds the array."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nq = off.size - 1
    h = _thresholds(H, nq)
    sc, _mat = make_scoring(scheme, index.alphabet)
    counts = np.zeros(max(nq, 1), dtype=np.int64)
    st = lib.ae_search_device_static(index.handle, ctypes.c_void_p(int(d_seq_ptr)), off.ctypes.data, nq,
                                     ctypes.byref(sc), h.ctypes.data,
                                     ctypes.byref(options) if options is not None else None,
                                     ctypes.c_void_p(int(d_hits_ptr)) if d_hits_ptr else None, int(capacity),
                                     counts.ctypes.data, _stream_handle(stream))
    if st not in (AE_OK, AE_EOVERFLOW, AE_EUNSUPPORTED):
        _check(st, "ae_search_device_static")
    return st, counts[:nq].copy()


def ae_hits_merge(d_hits_ptr, d_qid_ptr, n, nq, text_len, max_query_len, d_out_ptr, stream=None):
    """Per-cell maximum of n device result records (with device query ids) from
    partial searches. Returns (counts per query, total) of the records written
    to d_out (device, capacity n), grouped by query and sorted like ae_search."""
    counts = np.zeros(max(nq, 1), dtype=np.int64)
    total = ctypes.c_int64(0)
    _check(lib.ae_hits_merge(ctypes.c_void_p(int(d_hits_ptr)) if n else None,
                             ctypes.c_void_p(int(d_qid_ptr)) if n else None, int(n), int(nq), int(text_len),
                             int(max_query_len), ctypes.c_void_p(int(d_out_ptr)) if n else None,
                             counts.ctypes.data, ctypes.byref(total), _stream_handle(stream)), "ae_hits_merge")
    return counts[:nq].copy(), total.value


def ae_workspace_info(index, stream=None):
    """(bytes held by the workspace of `stream`, bytes held by all workspaces)."""
    b, t = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.ae_workspace_info(index.handle, _stream_handle(stream), ctypes.byref(b), ctypes.byref(t)),
           "ae_workspace_info")
    return b.value, t.value


def ae_workspace_release(index, stream=None):
    _check(lib.ae_workspace_release(index.handle, _stream_handle(stream)), "ae_workspace_release")


def ae_last_stats():
    s = ae_stats()
    _check(lib.ae_last_stats(ctypes.byref(s)), "ae_last_stats")
    d = {k: getattr(s, k) for k, _ in ae_stats._fields_}
    d["entries_tier"] = list(s.entries_tier)
    return d


def ae_suffix_array(codes, sigma):
    c = _u8(codes)
    sa = np.empty(c.size + 1, dtype=np.int32)
    _check(lib.ae_suffix_array(c.ctypes.data if c.size else None, c.size, int(sigma), sa.ctypes.data),
           "ae_suffix_array")
    return sa


def ae_suffix_array_device(d_codes_ptr, n, sigma, d_sa_ptr, reversed=False, stream=None):
    """Device suffix array: d_sa (n + 1 int32) of the n codes at d_codes
    (read backwards with `reversed`) plus the sentinel."""
    _check(lib.ae_suffix_array_device(d_codes_ptr or None, int(n), int(sigma), int(bool(reversed)), d_sa_ptr,
                                      _stream_handle(stream)), "ae_suffix_array_device")


def ae_plan(m, scheme, H, alphabet=AE_DNA):
    sc, _mat = make_scoring(scheme, alphabet)
    q = ctypes.c_int32()
    d0 = ctypes.c_int32()
    L = ctypes.c_int64()
    _check(lib.ae_plan(int(m), int(alphabet), ctypes.byref(sc), int(H), ctypes.byref(q), ctypes.byref(d0),
                       ctypes.byref(L)), "ae_plan")
    return q.value, d0.value, L.value


AE_PEAK_IADD, AE_PEAK_IMAX, AE_PEAK_ADDMAX32, AE_PEAK_ADDMAX16X2 = range(4)


def ae_int_peak(kind, chains=4, iters=2048, blocks_per_sm=8, stream=None):
    """Measured integer-ALU rate of one operation kind (include/ae_peak.h):
    (ops per second, instructions per second, kernel ms)."""
    ops, ins, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.ae_int_peak(int(kind), int(chains), int(iters), int(blocks_per_sm), _stream_handle(stream),
                           ctypes.byref(ops), ctypes.byref(ins), ctypes.byref(ms)), "ae_int_peak")
    return ops.value, ins.value, ms.value


def encode_codes(seq, alphabet=AE_DNA):
    """ASCII -> letter codes (host helper for tests of ae_suffix_array)."""
    a = np.frombuffer(ALPHABETS[alphabet], dtype=np.uint8)
    lut = np.full(256, 255, dtype=np.uint8)
    lut[a] = np.arange(a.size, dtype=np.uint8)
    c = lut[_u8(seq)]
    if c.size and c.max() == 255:
        raise ValueError("letter outside the alphabet")
    return c


# ------------------------------------------------------------------ work predictor (include/ae_mlp.h)

MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS = 66, 128, 2, 25346


class Mlp:
    """Owns one ae_mlp*.  Device arrays are passed as raw addresses (e.g. a
    torch tensor's data_ptr()); host arrays as numpy float32."""

    def __init__(self, seed=0):
        h = ctypes.c_void_p(0)
        _check(lib.ae_mlp_create(ctypes.c_uint64(seed), ctypes.byref(h)), "ae_mlp_create")
        self._h = h

    @property
    def handle(self):
        if not self._h:
            raise ValueError("model is closed")
        return self._h

    def close(self):
        if self._h:
            lib.ae_mlp_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if p.size != MLP_PARAMS:
            raise ValueError("wrong parameter count")
        _check(lib.ae_mlp_set_params(self.handle, p.ctypes.data), "ae_mlp_set_params")

    def get_params(self):
        p = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(lib.ae_mlp_get_params(self.handle, p.ctypes.data), "ae_mlp_get_params")
        return p

    def set_norm(self, x_mu, x_sd, y_mu, y_sd):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float32)) for a in (x_mu, x_sd, y_mu, y_sd)]
        _check(lib.ae_mlp_set_norm(self.handle, *[a.ctypes.data for a in arrs]), "ae_mlp_set_norm")

    def forward(self, d_x_ptr, B, d_y_ptr, stream=None):
        _check(lib.ae_mlp_forward(self.handle, ctypes.c_void_p(int(d_x_ptr)), int(B), ctypes.c_void_p(int(d_y_ptr)),
                                  _stream_handle(stream)), "ae_mlp_forward")

    def loss_grad(self, d_x_ptr, d_t_ptr, B, want_grads=True, stream=None):
        loss = ctypes.c_float(0)
        g = np.empty(MLP_PARAMS, dtype=np.float32) if want_grads else None
        _check(lib.ae_mlp_loss_grad(self.handle, ctypes.c_void_p(int(d_x_ptr)), ctypes.c_void_p(int(d_t_ptr)), int(B),
                                    ctypes.byref(loss), g.ctypes.data if g is not None else None,
                                    _stream_handle(stream)), "ae_mlp_loss_grad")
        return loss.value, g

    def train(self, d_x_ptr, d_t_ptr, n, epochs, batch, lr, weight_decay=0.0, seed=0, stream=None):
        loss = ctypes.c_float(0)
        _check(lib.ae_mlp_train(self.handle, ctypes.c_void_p(int(d_x_ptr)), ctypes.c_void_p(int(d_t_ptr)), int(n),
                                int(epochs), int(batch), ctypes.c_float(lr), ctypes.c_float(weight_decay),
                                ctypes.c_uint64(seed),
                                ctypes.byref(loss), _stream_handle(stream)), "ae_mlp_train")
        return loss.value


def ae_mlp_features(index, d_seq_ptr, offsets, d_feat_ptr, stream=None):
    """Features (nq x 66, device) of the queries in d_seq (device ASCII, back to
    back) delimited by offsets (host int64, nq+1)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nq = off.size - 1
    _check(lib.ae_mlp_features(index.handle, ctypes.c_void_p(int(d_seq_ptr)), off.ctypes.data, nq,
                               ctypes.c_void_p(int(d_feat_ptr)), _stream_handle(stream)), "ae_mlp_features")
