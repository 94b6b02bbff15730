"""Cloud-key checkpoint files: round trip, and corruption is detected."""
import numpy as np
import pytest

from paper_2506_12761_gb300 import keyfile, synth
from paper_2506_12761_gb300 import build
from paper_2506_12761_gb300 import velopir as vp


def test_round_trip_and_corruption(tmp_path):
    build.build()
    bk, ksk = vp.velopir_client_keygen(synth.key_material())
    p = tmp_path / "key.bin"
    keyfile.save_cloud_key(str(p), bk, ksk)
    bk2, ksk2 = keyfile.load_cloud_key(str(p))
    assert np.array_equal(bk, bk2) and np.array_equal(ksk, ksk2)
    raw = bytearray(p.read_bytes())
    raw[200000] ^= 1
    p.write_bytes(bytes(raw))
    with pytest.raises(ValueError, match="corrupt"):
        keyfile.load_cloud_key(str(p))
    p.write_bytes(bytes(raw[:1000]))
    with pytest.raises(ValueError, match="truncated"):
        keyfile.load_cloud_key(str(p))
    with pytest.raises(ValueError):
        keyfile.save_cloud_key(str(p), bk[:10], ksk)
