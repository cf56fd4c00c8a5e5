"""The C-ABI library builds, loads and exports every entry point declared in include/gs.h; host-side
argument checks reject bad calls before any launch (CPU only: no kernel runs here)."""
import ctypes
import os
import re

import pytest
import torch

from paper_2609_28458_gb300 import _abi, api
from paper_2609_28458_gb300 import build as gsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sysid_name = {v: k for k, v in _abi.SYSTEMS.items()}


@pytest.fixture(scope="module")
def lib():
    gsbuild.build()
    return _abi.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert set(names) == set(_abi.EXPORTS), names
    for n in names:
        assert hasattr(lib, n), n


def test_dims_and_defaults(lib):
    assert [_abi.dims(s) for s in ("isochrone", "mw", "precession", "quintessence", "loghalo")] == \
        [(6, 0), (6, 4), (9, 3), (3, 4), (6, 3)]
    o = _abi.options()
    assert (o.method, o.precision, o.max_steps, o.safety, o.alpha_min, o.alpha_max) == (0, 0, 1000000, 0.9, 0.2, 5.0)
    assert lib.gs_version().decode().startswith("gs-gb300")


def test_host_checks_reject_before_launch(lib):
    o = _abi.options()
    d, p = ctypes.c_int32(), ctypes.c_int32()
    assert lib.gs_dims(99, ctypes.byref(d), ctypes.byref(p)) == _abi.GS_ERR_INVALID
    assert "unknown system" in lib.gs_last_error().decode()
    # N = 0 is a valid no-op
    assert lib.gs_solve(0, 0, None, None, None, None, 1e-6, 1e-6, 0, None, ctypes.byref(o), None, None, None, None,
                        None, 0, None) == _abi.GS_OK
    # null inputs with N > 0
    assert lib.gs_solve(0, 4, None, None, None, None, 1e-6, 1e-6, 1, None, ctypes.byref(o), None, None, None, None,
                        None, 0, None) == _abi.GS_ERR_INVALID
    # bad tolerances / options
    fake = ctypes.c_void_p(256)
    assert lib.gs_solve(0, 4, fake, None, fake, fake, -1.0, 1e-6, 1, fake, ctypes.byref(o), fake, fake, fake, fake,
                        None, 0, None) == _abi.GS_ERR_INVALID
    o.method = 7
    assert lib.gs_solve(0, 4, fake, None, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, fake, fake,
                        None, 0, None) == _abi.GS_ERR_INVALID
    o = _abi.options(kernel="persistent")
    assert lib.gs_solve(0, 4, fake, None, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, fake, fake,
                        None, 0, None) == _abi.GS_ERR_WORKSPACE
    # vjp needs a tape workspace
    o = _abi.options()
    assert lib.gs_vjp(1, 4, fake, fake, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, fake, fake, fake,
                      fake, fake, None, 0, None) == _abi.GS_ERR_WORKSPACE


def test_workspace_sizes(lib):
    o = _abi.options()
    small = lib.gs_workspace_bytes(1, 1000, 1, ctypes.byref(o), 0, 0.0)
    big = lib.gs_workspace_bytes(1, 1000, 1, ctypes.byref(o), 1, 500.0)
    assert small >= 256 and big > small
    # a tape chunk holds 32 slots behind a 16-byte header; a slot is the state (8 d bytes in FP64,
    # 4 d for the FP32 high part), then the times: t, tc and the signed h as FP64 from the next
    # 8-byte boundary (24 bytes), or th, tl, h, flag as FP32 from the next 16-byte boundary (16 bytes,
    # FP32-pair mode); padded to 16 bytes
    assert (big - small) == (1000 * (16 + 1) + 1) * (16 + 32 * 80)
    for prec, word, fp32_tail in (("fp64", 8, False), ("fp32", 4, False), ("fp32df", 4, True)):
        o = _abi.options(precision=prec)
        for sysid, d in ((1, 6), (2, 9), (3, 3)):
            a = lib.gs_workspace_bytes(sysid, 1000, 1, ctypes.byref(o), 0, 0.0)
            b = lib.gs_workspace_bytes(sysid, 1000, 1, ctypes.byref(o), 1, 500.0)
            if fp32_tail:
                slot = (word * d + 15) // 16 * 16 + 16
            else:
                slot = ((word * d + 7) // 8 * 8 + 24 + 15) // 16 * 16
            assert slot % 16 == 0 and (b - a) == (1000 * (16 + 1) + 1) * (16 + 32 * slot)
            # the binding's exact sizing uses the same chunk size
            na = torch.full((1000,), 500, dtype=torch.int32)
            assert api.tape_bytes(sysid_name[sysid], 1000, n_accept=na, precision=prec) == a + (1000 * 16 + 1) * (16 + 32 * slot)


def test_solve_flat_argument_checks(lib):
    """gs_solve_flat rejects bad arguments on the host, before any launch."""
    o = _abi.options()
    fake = ctypes.c_void_p(256)
    ws_need = lib.gs_flat_workspace_bytes(1000, 8)
    assert ws_need >= 512 + 1000 * 8 * 3 * 2 * 8 + 1000 * 4 * 2 * 8 + 1000 * 4
    assert lib.gs_flat_workspace_bytes(10, 0) == 0 and lib.gs_flat_workspace_bytes(-1, 4) == 0

    def call(N=4, K=8, max_newton=8, gtol=1e-8, ws=fake, nbytes=1 << 30, opt=o):
        return lib.gs_solve_flat(N, fake, fake, fake, fake, 1e-6, 1e-9, K, fake, ctypes.byref(opt) if opt else None,
                                 max_newton, gtol, fake, None, None, None, fake, fake, fake, fake, ws, nbytes, None)

    assert call(K=0) == _abi.GS_ERR_INVALID
    assert call(max_newton=0) == _abi.GS_ERR_INVALID
    assert call(gtol=0.0) == _abi.GS_ERR_INVALID and call(gtol=float("nan")) == _abi.GS_ERR_INVALID
    assert call(opt=None) == _abi.GS_ERR_INVALID
    assert call(nbytes=1024) == _abi.GS_ERR_WORKSPACE
    assert call(ws=ctypes.c_void_p(8)) == _abi.GS_ERR_WORKSPACE
    assert call(N=0) == _abi.GS_OK


def test_order_option_checks(lib):
    """gs_options.order: unknown values, GS_ORDER_HINT without a hint and an explicit order without a
    workspace are rejected on the host."""
    fake = ctypes.c_void_p(256)
    for order, hint in ((7, None), (-1, None), (_abi.ORDERS["hint"], None)):
        o = _abi.options(kernel="plain", order=order)
        if hint is not None:
            o.cost_hint = hint
        rc = lib.gs_solve(0, 4, fake, None, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, fake, fake,
                          None, 0, None)
        assert rc == _abi.GS_ERR_INVALID, order
    # an explicit longest-first order without room for the work list fails; AUTO falls back to the
    # stored order (both before any device work)
    o = _abi.options(kernel="plain", order="estimate")
    rc = lib.gs_solve(0, 4, fake, None, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, fake, fake,
                      None, 0, None)
    assert rc == _abi.GS_ERR_WORKSPACE
    assert ctypes.sizeof(_abi.GsOptions) == 120


def test_checkpoint_stride_sizes_and_checks(lib):
    """gs_options.ckpt_stride: the chunk of a stride S > 1 holds 32 step lengths and 32 / S
    checkpoints (state, first stage and, in the FP32 modes, the state's low part; then the time);
    the part before the pool gains the int32 output attribution [N, K]; bad strides and the
    unsupported combinations are rejected on the host."""
    fake = ctypes.c_void_p(256)
    for prec, hbytes, words in (("fp64", 8, 4), ("fp32", 8, 3), ("fp32df", 4, 3)):
        for sysid, d in ((1, 6), (2, 9), (3, 3)):
            o1 = _abi.options(precision=prec)
            c1 = lib.gs_tape_chunk_bytes(sysid, ctypes.byref(o1))
            # steps_hint 1: one chunk per trajectory plus one, after the part before the pool
            assert lib.gs_workspace_bytes(sysid, 10, 1, ctypes.byref(o1), 1, 1.0) - \
                lib.gs_workspace_bytes(sysid, 10, 1, ctypes.byref(o1), 1, 0.0) == (10 * 2 + 1) * c1
            for S in (2, 4, 8, 16, 32):
                o = _abi.options(precision=prec, ckpt_stride=S)
                ck = (4 * words * d + 15) // 16 * 16 + 16
                assert lib.gs_tape_chunk_bytes(sysid, ctypes.byref(o)) == 16 + 32 * hbytes + (32 // S) * ck
                if S >= 4:  # (at S = 2 a checkpoint's low part and first stage outweigh the savings)
                    assert lib.gs_tape_chunk_bytes(sysid, ctypes.byref(o)) < c1
                K = 7
                a = lib.gs_workspace_bytes(sysid, 1000, K, ctypes.byref(o), 1, 0.0)
                assert a == lib.gs_workspace_bytes(sysid, 1000, K, ctypes.byref(o), 0, 0.0) + (1000 * K * 4 + 255) // 256 * 256
    # the Milky-Way FP32-pair tape at S = 16 is a fifth of S = 1's
    o1, o16 = _abi.options(precision="fp32df"), _abi.options(precision="fp32df", ckpt_stride=16)
    assert lib.gs_tape_chunk_bytes(1, ctypes.byref(o1)) / lib.gs_tape_chunk_bytes(1, ctypes.byref(o16)) > 4.5
    assert lib.gs_tape_chunk_bytes(1, ctypes.byref(_abi.options(ckpt_stride=3))) == 0
    assert lib.gs_tape_chunk_bytes(99, ctypes.byref(o1)) == 0

    def vjp(o):
        return lib.gs_vjp(0, 4, fake, None, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, None, fake,
                          fake, fake, fake, ctypes.c_void_p(1 << 20), 1 << 30, None)

    for bad in (3, -2, 64):
        assert vjp(_abi.options(ckpt_stride=bad)) == _abi.GS_ERR_INVALID
    assert vjp(_abi.options(ckpt_stride=8, kernel="plain")) == _abi.GS_ERR_INVALID
    assert "persistent" in lib.gs_last_error().decode()
    assert vjp(_abi.options(ckpt_stride=8, precision="df64")) == _abi.GS_ERR_INVALID
    # a workspace below the part before the pool plus one chunk is rejected for strides too
    o = _abi.options(ckpt_stride=8, kernel="persistent")
    need = lib.gs_workspace_bytes(0, 4, 1, ctypes.byref(o), 1, 0.0) + lib.gs_tape_chunk_bytes(0, ctypes.byref(o))
    rc = lib.gs_vjp(0, 4, fake, None, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake, None, fake, fake,
                    fake, fake, ctypes.c_void_p(1 << 20), need - 256, None)
    assert rc == _abi.GS_ERR_WORKSPACE


def test_noalloc_checks_the_system_first(lib):
    """An unknown system id is an invalid argument, not a scratch-size failure."""
    fake = ctypes.c_void_p(256)
    o = _abi.options()
    rc = lib.gs_vjp_noalloc(42, 1 << 30, fake, fake, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(o), fake, fake,
                            fake, fake, fake, fake, fake, None)
    assert rc == _abi.GS_ERR_INVALID and "unknown system" in lib.gs_last_error().decode()


def test_selftest_entry_checks_arguments_on_the_host(lib):
    """gs_selftest's check count matches the binding's, and bad arguments are refused before any CUDA
    call (the device run itself is tests/test_gpu_bits.py)."""
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    assert int(re.search(r"#define GS_SELFTEST_CHECKS (\d+)", src).group(1)) == _abi.SELFTEST_CHECKS
    from paper_2609_28458_gb300 import api
    assert len(api.SELFTEST_NAMES) == _abi.SELFTEST_CHECKS
    assert lib.gs_selftest(0, 0, None, None) == _abi.GS_ERR_INVALID
    assert lib.gs_selftest(16, 0, None, None) == _abi.GS_ERR_INVALID


def test_workspace_holds_the_prepared_starts(lib):
    """gs_workspace_bytes(for_vjp = 0) grows with N by the counters' 16 bytes plus a prepared-start row
    per trajectory for the persistent forward (112 to 256 bytes by system and precision; none in
    GS_DF64), and the part before the tape pool includes it."""
    for name, sysid in (("mw", 1), ("precession", 2), ("isochrone", 0)):
        for prec in ("fp64", "fp32", "fp32df"):
            o = _abi.options(precision=prec)
            a = lib.gs_workspace_bytes(sysid, 1 << 16, 1, ctypes.byref(o), 0, 0.0)
            b = lib.gs_workspace_bytes(sysid, 2 << 16, 1, ctypes.byref(o), 0, 0.0)
            per = (b - a) / float(1 << 16)
            assert 16 + 112 <= per <= 16 + 256, (name, prec, per)
            assert lib.gs_workspace_bytes(sysid, 1 << 16, 1, ctypes.byref(o), 1, 0.0) >= a
    o = _abi.options(precision="df64")
    a = lib.gs_workspace_bytes(0, 1 << 16, 1, ctypes.byref(o), 0, 0.0)
    b = lib.gs_workspace_bytes(0, 2 << 16, 1, ctypes.byref(o), 0, 0.0)
    assert (b - a) / float(1 << 16) == 16
