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
