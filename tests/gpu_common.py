"""Shared set-up of the GPU parity tests: one context with the cloud key made
by the library's own client code, and the oracle key from the same seed."""
import numpy as np

from paper_2506_12761_gb300 import build, synth
from paper_2506_12761_gb300 import velopir as vp

_state = {}


def gpu_ctx():
    if "ctx" not in _state:
        build.build()
        km = synth.key_material()
        bk, ksk = vp.velopir_client_keygen(km)
        ctx = vp.Context(0)
        vp.velopir_load_cloud_key(ctx.h, bk, ksk)
        vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
        _state.update(ctx=ctx, s=km.s.copy(), bk=bk, ksk=ksk)
    return _state["ctx"], _state["s"]


def encrypt_value_bits(s, value, width, seed):
    bits = synth.value_bits([value], width)[0]
    return vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(width, seed=seed))


def check_trace(keys, recs, min_records):
    """Recompute every traced gate with the oracle's linear gate from the
    recorded inputs and pre-combination; each output must be bit-identical.
    Returns the number of records checked."""
    import oracle
    assert len(recs) >= min_records, (len(recs), min_records)
    assert recs["nrot"].min() >= 1 and recs["nrot"].max() <= 2
    # nin = 0: a gate whose inputs are all trivial (e.g. the XOR of two zeroed payload bits)
    assert recs["nin"].max() <= vp.TRACE_MAX_IN
    want = oracle.gate_linear_batch(keys, recs["nrot"], recs["nin"], recs["coef"], recs["cst"], recs["ks_cst"],
                                    recs["inp"])
    bad = np.flatnonzero((want != recs["out"]).any(axis=1))
    assert bad.size == 0, f"{bad.size} of {len(recs)} traced gates differ from the oracle (first {bad[:5]})"
    return len(recs)


# ---- shared whole-circuit oracle runs --------------------------------------
# An interval-validation entry is 131 dependent bootstraps, so the oracle's
# whole IntV circuit takes the same wall time (about a minute on 16 cores)
# for one entry as for a dozen.  The IntV workloads that several GPU tests
# compare against the oracle (the two serving query sets, which the small
# whole-circuit tests reuse, and the sampled entries of the benchmark's
# D = 1,024 query) are therefore computed once, all at the same time.

def make_queries(s, seed, fanin=0):
    """IntV D=2 (the first rectangle contains the point), CoV D=3, IdM-8 D=4
    with payload (aggregated pairwise, or with fan-in `fanin`): three modes,
    uneven sizes."""
    qs = []
    w = synth.intv_workload(2, substream=seed)
    cx, cy = encrypt_value_bits(s, w["x"], 32, 900 + seed), encrypt_value_bits(s, w["y"], 32, 901 + seed)
    rects = np.ascontiguousarray(w["rects"], dtype=np.uint32)
    rects[0] = [max(0, w["x"] - 5), min(w["x"] + 5, 2 ** 32 - 1), max(0, w["y"] - 9), min(w["y"] + 1, 2 ** 32 - 1)]
    qs.append(dict(kind=vp.VP_QUERY_INTV, a=cx, b=cy, db=rects, D=2, out=np.zeros((2, 631), np.uint32), w=w))
    w = synth.cov_workload(3, substream=seed + 1)
    cell = encrypt_value_bits(s, w["cell"], 32, 902 + seed)
    qs.append(dict(kind=vp.VP_QUERY_COV, a=cell, db=w["cells"].astype(np.uint32), D=3,
                   out=np.zeros((3, 631), np.uint32), w=w))
    w = synth.idm_workload(4, 8, payload=True, substream=seed + 2)
    x = encrypt_value_bits(s, w["query"], 8, 903 + seed)
    qs.append(dict(kind=vp.VP_QUERY_IDM, a=x, db=w["ids"].astype(np.uint32), D=4, id_bits=8,
                   payload=w["payload"].astype(np.uint32), payload_bits=32, out=np.zeros((32, 631), np.uint32),
                   fanin=fanin, w=w))
    return qs


def as_record(q):
    return vp.make_query(q["kind"], q["a"], q["db"], q["D"], q["out"], enc_b=q.get("b"), id_bits=q.get("id_bits", 0),
                         payload=q.get("payload"), payload_bits=q.get("payload_bits", 0), agg_fanin=q.get("fanin", 0))


def fullsize_inputs(s):
    """The benchmark's query (IntV, D = 1,024) and the entries the oracle
    recomputes: the first two, the middle, the last and the first two hits."""
    D = 1024
    w = synth.intv_workload(D)
    cx = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["x"]], 32)[0], synth.lwe_material(32, substream=1))
    cy = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["y"]], 32)[0], synth.lwe_material(32, substream=2))
    rects = np.ascontiguousarray(w["rects"], dtype=np.uint32)
    r = rects.astype(np.int64)
    want = ((r[:, 0] <= w["x"]) & (w["x"] < r[:, 1]) & (r[:, 2] <= w["y"]) & (w["y"] < r[:, 3])).astype(np.uint32)
    sample = sorted({0, 1, D // 2, D - 1} | set(np.flatnonzero(want)[:2].tolist()))
    return dict(D=D, w=w, cx=cx, cy=cy, rects=rects, want=want, sample=sample)


def _qkey(q):
    return ("q", q["kind"], q["a"].tobytes(), q.get("fanin", 0))


def _oracle_circuit(keys, q):
    import oracle
    if q["kind"] == vp.VP_QUERY_INTV:
        return oracle.intv_batch(keys, q["a"], q["b"], q["db"].astype(np.uint64))
    if q["kind"] == vp.VP_QUERY_COV:
        return oracle.cov_batch(keys, q["a"], q["db"])
    return oracle.idm_payload(keys, q["a"], q["db"], q["payload"], q["payload_bits"], fanin=max(2, q.get("fanin", 0)))


_ORACLE = {}


def _shared_oracle_runs(keys):
    """The oracle's circuits for the serving query sets (seeds 3 and 4, the
    latter with fan-in 4) and for the benchmark query's sampled entries,
    computed once and concurrently."""
    if _ORACLE:
        return
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    _, s = gpu_ctx()
    qs = make_queries(s, 3) + make_queries(s, 4, fanin=4)
    f = fullsize_inputs(s)
    jobs = [(_qkey(q), (lambda q=q: _oracle_circuit(keys, q))) for q in qs]
    jobs.append((("fullsize",), lambda: oracle.intv_batch(keys, f["cx"], f["cy"],
                                                          f["rects"][f["sample"]].astype(np.uint64))))
    with ThreadPoolExecutor(len(jobs)) as ex:
        outs = list(ex.map(lambda j: j[1](), jobs))
    for (k, _), o in zip(jobs, outs):
        _ORACLE[k] = o


def oracle_out(keys, q):
    """The oracle's circuit for one query, from the query's own ciphertexts."""
    _shared_oracle_runs(keys)
    k = _qkey(q)
    if k not in _ORACLE:
        _ORACLE[k] = _oracle_circuit(keys, q)
    return _ORACLE[k]


def fullsize_oracle(keys):
    """The oracle's IntV circuit on fullsize_inputs()'s sampled entries."""
    _shared_oracle_runs(keys)
    return _ORACLE[("fullsize",)]
