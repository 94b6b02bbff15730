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
        _state.update(ctx=ctx, s=km.s.copy())
    return _state["ctx"], _state["s"]


def encrypt_value_bits(s, value, width, seed):
    bits = synth.value_bits([value], width)[0]
    return vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(width, seed=seed))
