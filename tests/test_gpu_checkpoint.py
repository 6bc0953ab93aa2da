"""States saved and restored bit for bit, and a 2D scan resumed from row-block
checkpoints after a deliberate interruption (host-side: the driver stops between
blocks, with no kernel in flight)."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2601_20550_gb300.heom")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(H.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


@pytest.mark.parametrize("precision", [0, 2])
def test_state_save_load_bit_exact(tmp_path, precision):
    model = W.small_three_mode(n=3, depth_L=2)
    h = H.heom_build_hierarchy(model, precision)
    rng = np.random.default_rng(8)
    shape = (2, h.n_ado, h.d, h.d)
    s = H.heom_state_create(h, 2, precision)
    H.heom_state_upload(s, rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    H.heom_propagate(h, s, 0.5, 3)
    p = str(tmp_path / "s.ckpt")
    H.heom_state_save(s, p)
    before = H.heom_state_download(s)
    t = H.heom_state_create(h, 2, precision)
    H.heom_state_load(t, p)
    # the same storage: the same download, and the same result after more steps
    assert np.array_equal(H.heom_state_download(t), before)
    H.heom_propagate(h, s, 0.5, 2)
    H.heom_propagate(h, t, 0.5, 2)
    assert np.array_equal(H.heom_state_download(t), H.heom_state_download(s))
    assert np.array_equal(H.heom_state_copy_out(t), H.heom_state_download(t))
    # a corrupted file leaves the target untouched; another shape is an argument error
    raw = bytearray(open(p, "rb").read())
    raw[200] ^= 0x40
    open(p, "wb").write(bytes(raw))
    keep = H.heom_state_download(t)
    with pytest.raises(H.HeomError) as ei:
        H.heom_state_load(t, p)
    assert ei.value.status == -8
    assert np.array_equal(H.heom_state_download(t), keep)
    H.heom_state_save(s, p)
    u = H.heom_state_create(h, 1, precision)
    with pytest.raises(H.HeomError) as ei:
        H.heom_state_load(u, p)
    assert ei.value.status == -1


def test_resumable_scan_matches_uninterrupted(tmp_path):
    from paper_2601_20550_gb300.resume import response_2d_resumable
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    grid = W.grid(0.5, 4, 7, 6, (0.0, 4.0), t_eq_fs=20.0)
    h = H.heom_build_hierarchy(model)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    d = str(tmp_path / "scan")
    with pytest.raises(StopIteration):
        response_2d_resumable(h, eq, grid, d, 3, stop_after=1)
    assert sorted(os.listdir(d)) == ["rows_0_3.ckpt"]
    # damage nothing yet: the resumed run reloads block 0 and computes the rest
    RI, RII, computed, reloaded = response_2d_resumable(h, eq, grid, d, 3)
    assert (computed, reloaded) == (2, 1)
    ri, rii = H.heom_response_2d_rows(h, eq, grid, 0, grid["n1"])
    assert np.array_equal(RI, ri) and np.array_equal(RII, rii)
    # a damaged block file is computed again, with the same result
    p = os.path.join(d, "rows_3_6.ckpt")
    raw = bytearray(open(p, "rb").read())
    raw[100] ^= 1
    open(p, "wb").write(bytes(raw))
    RI2, RII2, computed, reloaded = response_2d_resumable(h, eq, grid, d, 3)
    assert (computed, reloaded) == (1, 2)
    assert np.array_equal(RI2, ri) and np.array_equal(RII2, rii)
