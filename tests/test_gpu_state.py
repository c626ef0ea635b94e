"""Checkpoints of a run as bytes (sicp_export_state / sicp_import_state) and
resuming from them (sicp_resume), through the C ABI.  A run split at any
point, with its state exported, imported into another context and resumed,
returns the particles of the unsplit run bit for bit (same kernels, same
minibatch stream, same Adam step numbers).  The byte layout is checked
against its documented form with an independent CRC-32 (zlib's).
"""
import struct
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2106_03287_gb300 as S  # noqa: E402
from paper_2106_03287_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    from paper_2106_03287_gb300 import build
    build.build()
    a, b = S.sicp_create(0), S.sicp_create(0)
    yield a, b
    S.sicp_destroy(a)
    S.sicp_destroy(b)


@pytest.mark.parametrize("mode", [S.SICP_NN_GRID, S.SICP_NN_BRUTE_BF16, S.SICP_NN_GRID | S.SICP_INDEPENDENT])
def test_export_import_resume_equals_one_run(ctxs, mode):
    a, b = ctxs
    d = synth.make_box_problem(11, K=24)
    for c in (a, b):
        S.sicp_set_reference(c, d["ref"])
    par = lambda T: S.sicp_default_params(T=T, m=100, lr=0.01, seed=6, nn_mode=mode)  # noqa: E731
    full, mean_f, cov_f = S.sicp_register(a, d["src"], d["particles"], par(30))
    S.sicp_register(a, d["src"], d["particles"], par(12))
    blob = S.sicp_export_state(a)
    K = d["particles"].shape[0]
    assert len(blob) == 36 + 72 * K
    magic, version, k, t, seed = struct.unpack_from("<8sIiqQ", blob)
    assert (magic, version, k, t, seed) == (b"SICPRUN1", 1, K, 12, 6)
    assert struct.unpack_from("<I", blob, len(blob) - 4)[0] == zlib.crc32(blob[:-4])
    S.sicp_import_state(b, blob)
    th, mean, cov = S.sicp_resume(b, d["src"], par(18))
    assert np.array_equal(th, full)
    assert np.array_equal(mean, mean_f) and np.array_equal(cov, cov_f)
    # the resumed context's state has moved on to t = 30 and holds the final particles
    blob2 = S.sicp_export_state(b)
    assert struct.unpack_from("<q", blob2, 16)[0] == 30
    assert np.array_equal(np.frombuffer(blob2, np.float32, 6 * K, 32).reshape(K, 6), full)


def test_state_errors(ctxs):
    a, _ = ctxs
    fresh = S.sicp_create(0)
    try:
        with pytest.raises(S.SicpError) as e:        # no run yet
            S.sicp_export_state(fresh)
        assert e.value.code == S.SICP_EINVAL
        d = synth.make_box_problem(12, K=4)
        S.sicp_set_reference(a, d["ref"])
        S.sicp_register(a, d["src"], d["particles"], S.sicp_default_params(T=3, m=50, seed=2))
        blob = bytearray(S.sicp_export_state(a))
        for bad in (bytes(blob[:-1]), b"XXXXXXXX" + bytes(blob[8:]),
                    bytes(blob[:40]) + bytes([blob[40] ^ 1]) + bytes(blob[41:])):   # truncated, magic, checksum
            with pytest.raises(S.SicpError) as e:
                S.sicp_import_state(fresh, bad)
            assert e.value.code == S.SICP_EINVAL
        S.sicp_import_state(fresh, bytes(blob))
        S.sicp_set_reference(fresh, d["ref"])
        with pytest.raises(S.SicpError) as e:        # the run's minibatch stream is seed 2
            S.sicp_resume(fresh, d["src"], S.sicp_default_params(T=3, m=50, seed=3))
        assert e.value.code == S.SICP_EINVAL
    finally:
        S.sicp_destroy(fresh)
