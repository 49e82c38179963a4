"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/*.h declares; host-only calls work without a device."""
import ctypes

import numpy as np
import glob
import os
import re

import pytest

from paper_1910_13908_gb300 import build, sagecal

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names += re.findall(r"SC_API\s+[\w\s\*]+?\b(sc_\w+)\s*\(", open(h).read())
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for n in ("sc_predict_coherencies", "sc_residual", "sc_lm_normal_eqs", "sc_solve_cluster",
              "sc_calibrate_sage", "sc_workspace_size", "sc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    L = sagecal.lib()
    assert L.sc_version() >> 16 == 1
    # workspace sizing and argument checking need no device
    n = sagecal.workspace_size(sagecal.Shape(N=64, T=10, F=1, K=1, S_max=20), sagecal.SC_MIXED)
    assert n > 64 * 63 // 2 * 10 * 32
    with pytest.raises(sagecal.ScError) as e:
        sagecal.workspace_size(sagecal.Shape(N=1, T=10, F=1), sagecal.SC_MIXED)
    assert e.value.code == -1 and "N = 1" in str(e.value)
    with pytest.raises(sagecal.ScError):
        sagecal.workspace_size(sagecal.Shape(N=8, T=10, F=1), 7)


def test_residual_all_rejects_bad_arguments_before_touching_the_device(lib):
    # the pointers are never dereferenced: every check below fails first
    L = sagecal.lib()
    d = sagecal.Shape(N=8, T=2, F=3, K=4, S_max=1).c()
    fake = ctypes.c_void_p(1 << 20)
    for corr in (-2, 4, 100):
        rc = L.sc_residual_all(ctypes.byref(d), fake, fake, fake, corr, fake, None,
                               sagecal.SC_MIXED, fake, 1 << 30, None)
        assert rc == -1
        buf = ctypes.create_string_buffer(256)
        L.sc_last_error(buf, 256)
        assert b"corr = %d" % corr in buf.value
    rc = L.sc_residual_all(ctypes.byref(d), None, fake, fake, 0, fake, None, sagecal.SC_MIXED,
                           fake, 1 << 30, None)
    assert rc == -1
    rc = L.sc_residual_all(ctypes.byref(d), fake, fake, fake, 0, fake, None, 5, fake, 1 << 30, None)
    assert rc == -1


def test_calibrate_chunks_rejects_bad_arguments_before_touching_the_device(lib):
    L = sagecal.lib()
    d = sagecal.Shape(N=8, T=2, F=1, K=1, S_max=1).c()
    fake = ctypes.c_void_p(1 << 20)
    offs = (ctypes.c_int32 * 2)(0, 1)
    sky = sagecal.SkyC(offs, fake, fake, fake, fake, 150e6)
    opts = sagecal.SageOpts(1, sagecal.lm_opts())
    for n_chunks in (0, -3, 40000):
        rc = L.sc_calibrate_chunks(ctypes.byref(d), n_chunks, fake, fake, ctypes.byref(sky), fake, fake,
                                   None, ctypes.byref(opts), None, sagecal.SC_MIXED, fake, 1 << 30, None)
        assert rc == -1
        buf = ctypes.create_string_buffer(256)
        L.sc_last_error(buf, 256)
        assert b"n_chunks" in buf.value
    rc = L.sc_calibrate_chunks(ctypes.byref(d), 2, fake, fake, ctypes.byref(sky), None, fake, None,
                               ctypes.byref(opts), None, sagecal.SC_MIXED, fake, 1 << 30, None)
    assert rc == -1


def _documented_order(nT):
    """The factorisation list spelled out loop by loop: POTRF(0) and the
    TRSMs of column 0, then for each panel j the next column's updates,
    POTRF(j+1), the TRSMs of column j+1 and the remaining trailing updates."""
    out = [(0, 0, 0, 0)] + [(1, i, 0, 0) for i in range(1, nT)]
    for j in range(nT - 1):
        out += [(2, i, j + 1, j) for i in range(j + 1, nT)]
        out.append((0, j + 1, j + 1, j + 1))
        out += [(1, i, j + 1, j + 1) for i in range(j + 2, nT)]
        out += [(2, i, k, j) for k in range(j + 2, nT) for i in range(k, nT)]
    return out


def test_cholesky_task_decoder_matches_documented_order():
    """The closed-form decoder of list positions reproduces the documented
    loop order exactly, including orders far above the test sizes (the
    cube-root and quadratic estimates are corrected by exact comparisons)."""
    for nT in list(range(1, 40)) + [63, 64, 65, 100, 128, 129, 200]:
        assert [tuple(t) for t in sagecal.chol_schedule(nT, 0)] == _documented_order(nT), nT


def test_cholesky_task_order_respects_every_dependency():
    """Every task's inputs are produced by tasks earlier in the list, each
    tile receives its updates in panel order, and the list covers the
    right-looking factorisation exactly once (deadlock freedom of the
    persistent kernel rests on this)."""
    for nT in (1, 2, 3, 5, 8, 17):
        tasks = sagecal.chol_schedule(nT, 0)
        done_potrf, done_trsm, upd = set(), set(), {}
        seen = set()
        for typ, i, k, j in tasks:
            assert (typ, i, k, j) not in seen
            seen.add((typ, i, k, j))
            if typ == 0:
                assert upd.get((j, j), 0) == j
                done_potrf.add(j)
            elif typ == 1:
                assert i > j and j in done_potrf and upd.get((i, j), 0) == j
                done_trsm.add((i, j))
            else:
                assert i >= k > j
                assert (i, j) in done_trsm and (k, j) in done_trsm
                assert upd.get((i, k), 0) == j
                upd[(i, k)] = j + 1
        assert len(done_potrf) == nT
        assert len(done_trsm) == nT * (nT - 1) // 2
        assert sum(upd.values()) == sum(min(i, k) for i in range(nT) for k in range(i + 1))
        solve = sagecal.chol_schedule(nT, 1)
        assert [t[1] for t in solve] == list(range(nT)) + list(range(nT - 1, -1, -1))
        assert [t[0] for t in solve] == [3] * nT + [4] * nT


def test_graph_calls_reject_bad_arguments_before_touching_the_device(lib):
    # every check below fails before any CUDA call
    L = sagecal.lib()
    d = sagecal.Shape(N=8, T=2, F=3, K=1, S_max=1).c()
    fake = ctypes.c_void_p(1 << 20)
    o = sagecal.SageOpts(1, sagecal.lm_opts())
    h = ctypes.c_void_p(123)
    args = (ctypes.byref(d), fake, fake, None, fake, fake, ctypes.byref(o), None, sagecal.SC_MIXED, fake,
            1 << 30)
    assert L.sc_graph_capture_sage(*args, fake, None) == -1  # no place for the handle
    # the legacy default stream cannot be captured; the handle is cleared
    assert L.sc_graph_capture_sage(*args, None, ctypes.byref(h)) == -1
    assert h.value is None
    buf = ctypes.create_string_buffer(256)
    L.sc_last_error(buf, 256)
    assert b"legacy default stream" in buf.value
    assert L.sc_graph_launch(None, None) == -1
    assert L.sc_graph_destroy(None) == 0


def test_predict_full_rejects_bad_arguments_before_touching_the_device(lib):
    # the pointers are never dereferenced: every check below fails first
    L = sagecal.lib()
    fake = ctypes.c_void_p(1 << 20)

    def call(d, offsets, fields=None, f0=150e6, C=fake):
        offs = (ctypes.c_int32 * len(offsets))(*offsets)
        ptrs = [fake] * 10 if fields is None else fields
        sky = sagecal.SkyFullC(offs, *ptrs, f0)
        return L.sc_predict_coherencies_full(ctypes.byref(d), fake, fake, ctypes.byref(sky), C,
                                             sagecal.SC_MIXED, fake, 1 << 30, None)

    d = sagecal.Shape(N=8, T=2, F=3, K=2, S_max=4).c()
    assert call(d, [0, 2, 1]) == -1                       # offsets decrease
    assert call(d, [1, 2, 3]) == -1                       # offsets[0] != 0
    assert call(d, [0, 5, 6]) == -1                       # more sources than S_max
    assert call(d, [0, 2, 4], fields=[fake] * 9 + [None]) == -1   # a NULL source array
    assert call(d, [0, 2, 4], f0=0.0) == -1
    assert call(d, [0, 2, 4], C=None) == -1
    big = sagecal.Shape(N=8, T=1, F=40000, K=1, S_max=40000).c()
    assert call(big, [0, 1]) == -1                        # F * S_max > 2^30
    buf = ctypes.create_string_buffer(256)
    L.sc_last_error(buf, 256)
    assert b"F * S_max" in buf.value


def test_consensus_rejects_bad_arguments_before_touching_the_device(lib):
    # the pointers are never dereferenced: every check below fails first
    L = sagecal.lib()
    fake = ctypes.c_void_p(1 << 20)
    d = sagecal.Shape(N=8, T=2, F=3, K=2, S_max=4).c()
    offs = (ctypes.c_int32 * 3)(0, 2, 4)
    sky = sagecal.SkyC(offs, fake, fake, fake, fake, 150e6)

    def call(n_bands=4, n_poly=2, n_admm=2, rho=1.0, basis=fake, dual=fake, opts=True):
        o = sagecal.ConsensusOpts(sagecal.SageOpts(1, sagecal.lm_opts()), n_admm, n_poly, rho)
        return L.sc_calibrate_consensus(ctypes.byref(d), n_bands, fake, fake, ctypes.byref(sky), fake, basis,
                                        fake, dual, fake, None, ctypes.byref(o) if opts else None,
                                        sagecal.SC_MIXED, fake, 1 << 30, None)

    assert call(opts=False) == -1
    assert call(n_poly=0) == -1
    assert call(n_poly=9) == -1                           # at most 8 basis terms
    assert call(n_bands=1, n_poly=2) == -1                # fewer bands than basis terms
    assert call(n_bands=257) == -1                        # at most 256 bands
    assert call(n_admm=0) == -1
    assert call(rho=-1.0) == -1
    assert call(rho=float("nan")) == -1
    assert call(basis=None) == -1
    assert call(dual=None) == -1
    buf = ctypes.create_string_buffer(256)
    L.sc_last_error(buf, 256)
    assert b"must not be NULL" in buf.value


def test_lockstep_batch_task_list_keeps_each_jobs_dependencies_earlier():
    """The batched factorisation and solves take task t of a combined list as
    task t // G of job t % G.  Every job's dependencies then come earlier in
    the combined list, in the same relative order as in its own list, so the
    list-order argument against deadlock holds for the batch as well."""
    for nT, G in ((3, 2), (5, 3), (9, 5)):
        own = sagecal.chol_schedule(nT, 0)
        combined = [(t % G, own[t // G]) for t in range(len(own) * G)]
        for g in range(G):
            mine = [task for job, task in combined if job == g]
            assert mine == own
        # position of each job's task in the combined list grows with its own position
        pos = {}
        for t, (g, task) in enumerate(combined):
            pos[(g, tuple(task))] = t
        for g in range(G):
            order = [pos[(g, tuple(task))] for task in own]
            assert order == sorted(order)


def test_batched_workspace_size_is_host_only(lib):
    L = sagecal.lib()
    dims = (sagecal.Dims * 3)(sagecal.Shape(70, 3, 2, 2, 5).c(), sagecal.Shape(70, 9, 1, 2, 4).c(),
                               sagecal.Shape(70, 1, 4, 2, 6).c())
    n3 = ctypes.c_size_t(0)
    assert L.sc_batched_workspace_size(dims, 3, sagecal.SC_MIXED, ctypes.byref(n3)) == 0
    one = (sagecal.Dims * 1)(sagecal.Shape(70, 9, 1, 2, 4).c())
    n1 = ctypes.c_size_t(0)
    assert L.sc_batched_workspace_size(one, 1, sagecal.SC_MIXED, ctypes.byref(n1)) == 0
    # one block per job, each sized for the largest job's statistics, then
    # the merged task order (4 bytes per factorisation task of every job)
    tasks = len(sagecal.chol_schedule((8 * 70 + 63) // 64, 0))
    a256 = lambda x: (x + 255) // 256 * 256
    block = n1.value - a256(4 * tasks)
    assert n3.value == 3 * block + a256(3 * 4 * tasks)
    P = 8 * 70
    assert n1.value > 4 * P * P                      # the float32 matrix of one job
    bad = (sagecal.Dims * 2)(sagecal.Shape(70, 3, 2, 2, 5).c(), sagecal.Shape(71, 3, 2, 2, 5).c())
    assert L.sc_batched_workspace_size(bad, 2, sagecal.SC_MIXED, ctypes.byref(n3)) == -1
    assert L.sc_batched_workspace_size(bad, 0, sagecal.SC_MIXED, ctypes.byref(n3)) == -1


def test_staggered_batch_order_is_a_permutation_keeping_each_jobs_order(lib):
    """The staggered merge of the jobs' factorisation lists (positions from
    the closed form the device kernel uses) fills every slot exactly once,
    keeps each job's own order (so dependencies stay earlier: no deadlock),
    and with window W has job g start after job g - W has done most of its
    list."""
    for nT, G, W in ((1, 1, 1), (3, 2, 1), (5, 3, 2), (9, 7, 3), (9, 7, 7), (17, 5, 64), (32, 64, 6)):
        pos = sagecal.batch_order(nT, G, W)
        n = pos.shape[1]
        assert sorted(pos.ravel().tolist()) == list(range(n * G)), (nT, G, W)
        assert np.all(np.diff(pos, axis=1) > 0)
        if G > W:
            # job W starts only after the whole of job 0: about W jobs in flight
            assert int(np.sum(pos[0] < pos[W, 0])) == n
        if G > 1:
            # job 1 starts once job 0 is a fraction 1 / W through its list
            assert int(np.sum(pos[0] < pos[1, 0])) == min(n, 1 + n // W)
