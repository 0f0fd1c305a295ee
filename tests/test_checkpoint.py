"""Checkpoint files: gauge field, sources and network parameters with a
header (host logic; the GPU round trip of a trained network is in
test_gpu_cnn.py)."""
import numpy as np
import pytest

from paper_1009_5169_gb300 import checkpoint, inputs


def test_round_trip_is_exact(tmp_path):
    U = inputs.links(4, 5, 0.3, 7)
    phi = inputs.sources(4, 5, 3, 8)
    params = np.random.default_rng(9).standard_normal(1234).astype(np.float32)
    meta = {"L": 4, "T": 5, "kappa": 0.13, "seed_links": 7, "epoch": 12}
    p = tmp_path / "c.npz"
    checkpoint.save(str(p), links=U, sources=phi, cnn_hidden=16, cnn_params=params, meta=meta)
    c = checkpoint.load(str(p))
    assert c["meta"] == meta and c["cnn_hidden"] == 16
    assert c["links"].dtype == np.complex128 and np.array_equal(c["links"], U)
    assert np.array_equal(c["sources"], phi)
    assert c["cnn_params"].dtype == np.float32 and np.array_equal(c["cnn_params"], params)


def test_partial_checkpoint_and_errors(tmp_path):
    p = tmp_path / "links_only.npz"
    U = inputs.links(4, 3, 0.2, 1)
    checkpoint.save(str(p), links=U)
    c = checkpoint.load(str(p))
    assert set(c) == {"meta", "cnn_hidden", "links"} and c["cnn_hidden"] is None
    with pytest.raises(ValueError):
        checkpoint.save(str(tmp_path / "x.npz"), cnn_params=np.zeros(3, np.float32))
    q = tmp_path / "other.npz"
    np.savez(str(q), links=U)
    with pytest.raises(ValueError):
        checkpoint.load(str(q))
    with pytest.raises(ValueError):
        checkpoint.load_cnn(str(p))
