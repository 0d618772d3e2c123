"""State dump/restore round trip (host only)."""
import numpy as np
import pytest

from paper_2602_21644_gb300 import state, synth


def test_round_trip(tmp_path):
    sc = synth.tiny_scene(3)
    blob, master = synth.mpnet_init(2)
    adam = np.arange(13, dtype=np.float64)
    p = str(tmp_path / "s.npz")
    state.save_state(p, seeds={"scene": 3, "net": 2}, gauss=sc.records, poses=sc.poses, adam=adam, blob=blob,
                     master=master, labels=np.zeros(5, np.uint8))
    arrays, seeds = state.load_state(p)
    assert seeds == {"scene": 3, "net": 2}
    np.testing.assert_array_equal(arrays["gauss"], sc.records)
    np.testing.assert_array_equal(arrays["poses"], sc.poses)
    np.testing.assert_array_equal(arrays["adam"], adam)
    np.testing.assert_array_equal(arrays["blob"], blob)
    assert arrays["gauss"].dtype == np.float32 and arrays["labels"].dtype == np.uint8


def test_torch_tensors_and_bad_file(tmp_path):
    torch = pytest.importorskip("torch")
    p = str(tmp_path / "t.npz")
    state.save_state(p, x=torch.arange(4, dtype=torch.float64))
    arrays, _ = state.load_state(p)
    np.testing.assert_array_equal(arrays["x"], np.arange(4.0))
    q = str(tmp_path / "bad.npz")
    np.savez(q, a=np.zeros(2))
    with pytest.raises(Exception):
        state.load_state(q)
