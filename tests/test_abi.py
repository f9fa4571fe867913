"""The C ABI library builds, loads and exports every entry point declared in
include/extconv.h (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "extconv.h")).read()
    return sorted(set(re.findall(r"\b(ext_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    from paper_2006_13188_gb300 import EXPORTED
    assert sorted(EXPORTED) == declared_symbols()


def test_library_exports_every_declared_symbol():
    from paper_2006_13188_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    from paper_2006_13188_gb300 import lib
    L = lib()
    assert L.ext_status_string(0) == b"EXT_OK"
    assert L.ext_status_string(2) == b"EXT_ERR_UNSUPPORTED"


def test_selection_rule_in_the_library_matches_the_oracle():
    """ext_select_components (host only) against the oracle's rule on random
    energies, with ties and budgets beyond K + 1."""
    import numpy as np
    from oracle.selection import select_components
    from paper_2006_13188_gb300 import ExtError, ext_select_components
    rng = np.random.default_rng(5)
    for K in (0, 1, 4, 16):
        E = rng.random(K + 1)
        if K >= 4:
            E[2] = E[3]                      # a tie: the smaller k first
        for budget in range(1, K + 4):
            assert ext_select_components(E, budget) == select_components(E, budget), (K, budget)
    with pytest.raises(ExtError) as e:
        ext_select_components(np.array([1.0, np.nan]), 2)
    assert e.value.status == 1
    with pytest.raises(ExtError):
        ext_select_components(np.array([1.0, 2.0]), 0)


def _checkpoint_bytes(n_in, hidden, step, rng):
    """A checkpoint written from its documented layout (independently of the
    library's writer), with zlib's CRC-32 of IEEE 802.3."""
    import struct
    import zlib
    import numpy as np
    n = hidden * (n_in + hidden + 6) + 4
    head = b"EXTMLP01" + struct.pack("<IIII", 1, n_in, hidden, 0) + struct.pack("<QQ", step, n)
    body = rng.standard_normal(3 * n).astype("<f4").tobytes()
    data = head + body
    return data + struct.pack("<I", zlib.crc32(data) & 0xFFFFFFFF)


def test_checkpoint_check_without_gpu(tmp_path):
    """ext_mlp_checkpoint_info accepts a well-formed file and rejects a
    flipped byte, a truncated file, a wrong magic, an impossible header and a
    missing file with EXT_ERR_CHECKPOINT (host only)."""
    import numpy as np
    from paper_2006_13188_gb300 import ExtError, ext_mlp_checkpoint_info
    rng = np.random.default_rng(9)
    good = _checkpoint_bytes(35, 32, 1234, rng)
    p = tmp_path / "net.ckpt"
    p.write_bytes(good)
    assert ext_mlp_checkpoint_info(p) == (35, 32, 1234)
    bad_cases = {
        "flipped": bytearray(good),
        "truncated": good[:-100],
        "magic": b"EXTMLP02" + good[8:],
        "header": good[:12] + (17).to_bytes(4, "little") + good[16:],
    }
    bad_cases["flipped"][len(good) // 2] ^= 0x10
    for name, data in bad_cases.items():
        q = tmp_path / f"{name}.ckpt"
        q.write_bytes(bytes(data))
        with pytest.raises(ExtError) as e:
            ext_mlp_checkpoint_info(q)
        assert e.value.status == 6, name
    with pytest.raises(ExtError) as e:
        ext_mlp_checkpoint_info(tmp_path / "missing.ckpt")
    assert e.value.status == 6
