"""Rows of A replaced between iterations (a time-dependent matrix, Eq. 1;
the data update step of Section 3) against the FP64 oracle through the C
ABI: stored values, norms and records of the new rows, one-step parity,
trajectories with the whole matrix changing at every tick, per-row
rejection of invalid rows."""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import nsli, workloads

pytestmark = pytest.mark.gpu

STORAGES = ["f64", "f32", "bf16", "fp8"]


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def stored_values(A32, storage):
    if storage == "bf16":
        return oracle.quantize_bf16(A32)
    if storage == "fp8":
        q, _ = oracle.quantize_e4m3_rows(A32)
        return q
    return A32


def src(A32, storage):
    return A32.astype(np.float64) if storage == "f64" else A32


@pytest.mark.parametrize("storage", STORAGES)
def test_updated_rows_equal_created_rows(storage):
    """A handle created on A and updated to A' row block by row block (host
    and device sources, with new b0) holds exactly what a handle created on
    A' holds: stored values, norms, and one Map/Reduce."""
    import torch
    m, n = 1500, 700
    p = workloads.dense_system(m, n, seed=61)
    q = workloads.dense_system(m, n, seed=62)
    with nsli.Solver(src(p["A"], storage), p["b0"], p["x0"], Av=p["Av"], storage=storage) as s, \
            nsli.Solver(src(q["A"], storage), q["b0"], p["x0"], Av=p["Av"], storage=storage) as t:
        s.update_rows(0, src(q["A"][:600], storage), b0=q["b0"][:600])             # host rows
        dev = torch.from_numpy(src(q["A"][600:], storage)).cuda()
        s.update_rows(600, dev, b0=torch.from_numpy(q["b0"][600:]).cuda())      # device rows
        np.testing.assert_array_equal(s.stored_rows(), t.stored_rows())
        np.testing.assert_array_equal(s.stored_rows(), stored_values(q["A"], storage).astype(np.float64))
        np.testing.assert_array_equal(s.norms2(), t.norms2())
        ys, hs, sts = s.map_reduce()
        yt, ht, stt = t.map_reduce()
        np.testing.assert_array_equal(ys, yt)
        assert hs == ht and sts == stt


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_trajectory_with_matrix_changing_every_tick(storage):
    """Every entry of A changes before every iteration (c_u = (n + 1) m,
    Section 4): every step matches the oracle's step on A(k) from the same
    x_k element by element, and the iterates match the oracle run on the
    same A(k) sequence until the first ambiguous row."""
    m, n, K = 900, 240, 10
    p = workloads.dense_system(m, n, seed=63)
    tol = 1e-12 if storage == "f64" else 1e-5
    x = p["x0"].copy()
    compared = 0
    together = True
    with nsli.Solver(src(p["A"], storage), p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        for k in range(K):
            Ak = workloads.drifted_matrix(p["A"], k, seed=64)
            s.update_rows(0, src(Ak, storage))
            A64 = Ak.astype(np.float64)
            n2, _ = oracle.norms2(A64)
            np.testing.assert_allclose(s.norms2(), n2, rtol=1e-13)
            code, x_next, st, y, r = oracle.iteration(A64, p["b0"], p["Av"], 1e-3, k, n2, x)
            xg = s.get_x()
            drift = np.linalg.norm(xg - x)
            u = 2.0 ** -53 if storage == "f64" else 2.0 ** -24
            bound = 64 * u * (np.abs(A64) @ np.abs(x) + np.abs(p["b0"]) + 1.0) + np.sqrt(n2) * drift * 1.01
            together = together and not np.any(np.abs(r) <= bound)
            s.iterate(1, rho=1e-3)
            x1 = s.get_x()
            # the step from the device's own x_k on A(k), element by element
            parity.check_step(xg, x1, None, A64, oracle.tick_b(p["b0"], p["Av"], 1e-3, k),
                              storage, depth=parity.dense_y_depth(m, parity.num_sms()), n2=n2,
                              levels=parity.dot_levels(n))
            if together:
                x = x_next
                rel = np.linalg.norm(x1 - x) / np.linalg.norm(x)
                assert rel <= tol, (k, rel)
                compared += 1
    assert compared >= 3


def test_invalid_rows_are_rejected_one_by_one():
    m, n = 300, 50
    p = workloads.dense_system(m, n, seed=65)
    new = workloads.dense_system(m, n, seed=66)["A"][:10].copy()
    new[3, 7] = np.nan
    new[5, :] = 0.0
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"]) as s:
        before = s.stored_rows()
        with pytest.raises(nsli.NsliError) as e:
            s.update_rows(20, new)
        assert e.value.code in (nsli.ERR_NONFINITE, nsli.ERR_ZERO_ROW)
        after = s.stored_rows()
        for q in range(10):
            want = before[20 + q] if q in (3, 5) else new[q].astype(np.float64)
            np.testing.assert_array_equal(after[20 + q], want)
        np.testing.assert_array_equal(after[:20], before[:20])
        np.testing.assert_array_equal(after[30:], before[30:])
        # the handle still iterates on the valid system
        s.iterate(3)
        assert np.all(np.isfinite(s.get_x()))
        with pytest.raises(nsli.NsliError) as e:
            s.update_rows(5, new[5:6])
        assert e.value.code == nsli.ERR_ZERO_ROW
        with pytest.raises(nsli.NsliError) as e:
            s.update_rows(295, new[:10])
        assert e.value.code == nsli.ERR_ARG


def test_update_rows_on_sparse_handle_unsupported():
    p = workloads.sparse_system(100, 40, 4, seed=67)
    with nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"], p["x0"]) as s:
        with pytest.raises(nsli.NsliError) as e:
            s.update_rows(0, np.ones((1, 40), np.float32))
        assert e.value.code == nsli.ERR_UNSUPPORTED


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("n, pad", [(1024, 0), (1027, 1), (20000, 0), (30000, 0)])
def test_staged_and_global_update_paths_agree(storage, n, pad, monkeypatch):
    """Rows short enough for shared memory and 16-byte aligned are staged
    there by one bulk copy (with a ragged tail when n * 4 is not a multiple
    of 16: n = 1027 from a source of pitch 1028); longer ones (n = 30000
    from binary32, n >= 20000 from binary64) and FP8 rows read global
    memory.  Either way the updated rows equal rows created from the same
    values, bit for bit, and the two paths give the same stored values and
    norms."""
    import ctypes
    import torch
    m = 48
    p = workloads.dense_system(m, n, seed=71)
    q = workloads.dense_system(m, n, seed=72)
    lib = nsli.load()
    srcq = src(q["A"], storage)
    dev = torch.zeros((m, n + pad), dtype=torch.float64 if storage == "f64" else torch.float32,
                      device="cuda")
    dev[:, :n] = torch.from_numpy(srcq).cuda()
    a_dtype = nsli.F64 if storage == "f64" else nsli.F32
    torch.cuda.synchronize()
    results = []
    with nsli.Solver(srcq, q["b0"], p["x0"], Av=p["Av"], storage=storage) as t:
        want_rows, want_n2 = t.stored_rows(), t.norms2()
        for staged in ("1", "0"):
            monkeypatch.setenv("NSLI_UPDATE_STAGED", staged)
            with nsli.Solver(src(p["A"], storage), q["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
                rc = lib.nsli_update_rows(s._h, 0, m, a_dtype, ctypes.c_void_p(dev.data_ptr()), n + pad, None)
                assert rc == nsli.OK
                rows, n2 = s.stored_rows(), s.norms2()
                np.testing.assert_array_equal(rows, want_rows)
                np.testing.assert_array_equal(n2, want_n2)
                ys, hs, sts = s.map_reduce()
                yt, ht, stt = t.map_reduce()
                np.testing.assert_array_equal(ys, yt)
                assert hs == ht and sts == stt
                results.append((rows, n2))
    np.testing.assert_array_equal(results[0][0], results[1][0])
    np.testing.assert_array_equal(results[0][1], results[1][1])


def test_bf16_rounding_of_created_and_updated_rows_at_the_edges():
    """bf16 storage rounds to nearest, ties to even, in the set-up and the
    row-update kernels alike (the scalar and the paired conversion): ties of
    both parities,
    subnormal values and ties, signed zeros and values next to the largest
    bf16 are stored as the oracle's rounding gives them, whether the row was
    created or updated; a value that rounds to infinity makes its row
    invalid in both."""
    import torch
    n = 2048
    rng = np.random.default_rng(81)
    base = (np.arange(1, 513, dtype=np.uint32) << np.uint32(16)) | np.uint32(0x3f800000)
    ties = (base + np.uint32(0x8000)).view(np.float32)              # halfway, both parities
    sub = ((np.arange(1, 257, dtype=np.uint32) << np.uint32(16)) + np.uint32(0x8000)).view(np.float32)
    near = np.array([3.3895314e38, -3.3895314e38, 3.38e38, 1.17549435e-38, -1.17549435e-38,
                     1e-40, -1e-40, 0.0, -0.0, 1.0], np.float32)
    rows = np.zeros((8, n), np.float32)
    rows[0, :512] = ties
    rows[1, :512] = -ties
    rows[2, :256] = sub
    rows[2, 256] = 1.0
    rows[3, :256] = -sub
    rows[3, 256] = -1.0
    rows[4, :10] = near
    rows[5:] = rng.standard_normal((3, n)).astype(np.float32)
    p = workloads.dense_system(8, n, seed=82)
    want = oracle.quantize_bf16(rows).astype(np.float64)
    with nsli.Solver(rows, p["b0"], p["x0"], storage="bf16") as t:
        np.testing.assert_array_equal(t.stored_rows(), want)
        n2_created = t.norms2()
    with nsli.Solver(p["A"], p["b0"], p["x0"], storage="bf16") as s:
        s.update_rows(0, torch.from_numpy(rows).cuda())
        np.testing.assert_array_equal(s.stored_rows(), want)
        np.testing.assert_array_equal(s.norms2(), n2_created)
        before = s.stored_rows()
        bad = rows[5:6].copy()
        bad[0, 3] = 3.4e38                                           # rounds to infinity in bf16
        with pytest.raises(nsli.NsliError) as e:
            s.update_rows(5, torch.from_numpy(bad).cuda())
        assert e.value.code == nsli.ERR_NONFINITE
        np.testing.assert_array_equal(s.stored_rows(), before)
    with pytest.raises(nsli.NsliError) as e:
        bad_all = rows.copy()
        bad_all[6, 3] = 3.4e38
        nsli.Solver(bad_all, p["b0"], p["x0"], storage="bf16")
    assert e.value.code == nsli.ERR_NONFINITE


def test_fp8_rounding_of_created_and_updated_rows_at_the_edges():
    """FP8 E4M3 storage (per-row power-of-two scales) rounds to nearest, ties
    to even, in the set-up and the row-update kernels alike: every value
    halfway between two neighbouring codes, normal and subnormal, both
    signs, the codes themselves and signed zeros are stored as the oracle's
    rounding gives them."""
    import torch
    n = 1024
    codes = np.arange(0, 0x7E, dtype=np.uint32)

    def decode(c):
        e = (c >> 3) & 0xF
        m = c & 7
        return np.where(e == 0, m * 2.0 ** -9, (1 + m / 8.0) * 2.0 ** (e.astype(np.int64) - 7))

    v0, v1 = decode(codes), decode(codes + 1)
    ties = ((v0 + v1) / 2).astype(np.float32)
    rows = np.zeros((6, n), np.float32)
    for r, vals in enumerate([ties, -ties, v0.astype(np.float32), -v0.astype(np.float32)]):
        rows[r, :vals.size] = vals
        rows[r, n - 1] = 448.0          # row scale 1: the values are the codes' own
    rows[4, :4] = [0.0, -0.0, 448.0, -2.0 ** -9]
    rows[4, 4:] = np.random.default_rng(83).standard_normal(n - 4).astype(np.float32) * 1e-3
    rows[5] = np.random.default_rng(84).standard_normal(n).astype(np.float32) * 37.0
    want, _ = oracle.quantize_e4m3_rows(rows)
    p = workloads.dense_system(6, n, seed=85)
    with nsli.Solver(rows, p["b0"], p["x0"], storage="fp8") as t:
        np.testing.assert_array_equal(t.stored_rows(), want.astype(np.float64))
        n2_created = t.norms2()
        yt, ht, stt = t.map_reduce()
    with nsli.Solver(p["A"], p["b0"], p["x0"], storage="fp8") as s:
        s.update_rows(0, torch.from_numpy(rows).cuda())
        np.testing.assert_array_equal(s.stored_rows(), want.astype(np.float64))
        np.testing.assert_array_equal(s.norms2(), n2_created)
        ys, hs, sts = s.map_reduce()
    np.testing.assert_array_equal(ys, yt)
    assert hs == ht and sts == stt
