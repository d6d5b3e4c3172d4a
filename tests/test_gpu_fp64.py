"""GPU parity of the plain FP64 out-of-core path against the CPU oracle.

All calls go through the C ABI (libooc.so) with pinned host operands; the
oracle computes the same product in FP64 on the CPU.  Tolerance for the plain
form: relative Frobenius error <= 1e-13 (two FP64 summation orders differ by
about sqrt(K) * 2^-53 relative); integer-valued inputs must match bit for bit.
"""
import itertools
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import np64, pinned, pinned_from

pytestmark = pytest.mark.gpu
TOL = 1e-13


def run_dgemm(P, ta, tb, A, B, C, alpha, beta, budget, opts=None):
    M = A.shape[0] if ta == "N" else A.shape[1]
    K = A.shape[1] if ta == "N" else A.shape[0]
    N = B.shape[1] if tb == "N" else B.shape[0]
    st = P.ooc_stats()
    lda = A.stride(0) if A.shape[0] > 1 else max(1, A.shape[1])
    ldb = B.stride(0) if B.shape[0] > 1 else max(1, B.shape[1])
    ldc = C.stride(0) if C.shape[0] > 1 else max(1, C.shape[1])
    rc = P.ooc_dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, budget, opts, st)
    return rc, st


def test_config_small_full_matrix(ooc):
    """1024^3, U[-1,1], alpha 1, beta 0, 4 MB budget: at least 8 C blocks stream."""
    n = 1024
    A = pinned_from(1, 0, n, n, synth.UNIFORM)
    B = pinned_from(1, 1, n, n, synth.UNIFORM)
    C = pinned(n, n, fill=np.nan)
    rc, st = run_dgemm(ooc, "N", "N", A, B, C, 1.0, 0.0, 4 << 20)
    assert rc == 0, ooc.ooc_last_error()
    assert st.steps >= 8 and st.blocks >= 2 and st.device_bytes <= 4 << 20
    ref = oracle.gemm("N", "N", 1.0, np64(A), np64(B), 0.0, None)
    assert oracle.rel_fro(np64(C), ref) <= TOL


def test_integer_inputs_are_exact(ooc):
    M, N, K = 700, 500, 900
    A = pinned_from(2, 0, M, K, synth.INTEGER, 1024)
    B = pinned_from(2, 1, K, N, synth.INTEGER, 1024)
    C = pinned_from(2, 2, M, N, synth.INTEGER, 1024)
    C0 = np64(C)
    rc, st = run_dgemm(ooc, "N", "N", A, B, C, 2.0, -3.0, 1 << 20)
    assert rc == 0, ooc.ooc_last_error()
    ref = oracle.gemm("N", "N", 2.0, np64(A), np64(B), -3.0, C0)
    assert np.array_equal(np64(C), ref)


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_transposes_ragged_padded(ooc, ta, tb):
    M, N, K = 300, 200, 170
    sa = (M, K) if ta == "N" else (K, M)
    sb = (K, N) if tb == "N" else (N, K)
    A = pinned_from(3, 0, *sa, synth.NORMAL, ld=sa[1] + 5)
    B = pinned_from(3, 1, *sb, synth.NORMAL, ld=sb[1] + 3)
    C = pinned_from(3, 2, M, N, synth.NORMAL, ld=N + 7)
    C0 = np64(C)
    opts = ooc.make_opts(mb=64, nb=64, kb=64, depth=2, c_buffers=2)
    rc, st = run_dgemm(ooc, ta, tb, A, B, C, 1.5, 0.5, 1 << 30, opts)
    assert rc == 0, ooc.ooc_last_error()
    assert st.steps == 5 * 4 * 3
    ref = oracle.gemm(ta, tb, 1.5, np64(A), np64(B), 0.5, C0)
    assert oracle.rel_fro(np64(C), ref) <= TOL


def test_auto_plan_tiny_budget_many_blocks(ooc):
    M, N, K = 1000, 700, 300
    A = pinned_from(4, 0, M, K, synth.UNIFORM)
    B = pinned_from(4, 1, K, N, synth.UNIFORM)
    C = pinned_from(4, 2, M, N, synth.UNIFORM)
    C0 = np64(C)
    rc, st = run_dgemm(ooc, "N", "N", A, B, C, -1.0, 2.0, 512 << 10)
    assert rc == 0, ooc.ooc_last_error()
    assert st.device_bytes <= 512 << 10 and st.blocks > 1
    ref = oracle.gemm("N", "N", -1.0, np64(A), np64(B), 2.0, C0)
    assert oracle.rel_fro(np64(C), ref) <= TOL


def test_beta_zero_ignores_nan_and_alpha_zero(ooc):
    M, N, K = 130, 250, 90
    A = pinned_from(5, 0, M, K, synth.UNIFORM)
    B = pinned_from(5, 1, K, N, synth.UNIFORM)
    C = pinned(M, N, fill=np.nan)
    rc, _ = run_dgemm(ooc, "N", "N", A, B, C, 1.0, 0.0, 1 << 20)
    assert rc == 0 and np.isfinite(np64(C)).all()
    assert oracle.rel_fro(np64(C), oracle.gemm("N", "N", 1.0, np64(A), np64(B), 0.0, None)) <= TOL
    C2 = pinned_from(5, 2, M, N, synth.UNIFORM)
    C20 = np64(C2)
    rc, _ = run_dgemm(ooc, "N", "N", A, B, C2, 0.0, 0.5, 1 << 20)
    assert rc == 0 and np.array_equal(np64(C2), 0.5 * C20)


def test_k_zero_scales_c(ooc):
    M, N = 77, 45
    A = pinned(M, 1)
    B = pinned(1, N)
    C = pinned_from(6, 2, M, N, synth.NORMAL)
    C0 = np64(C)
    st = ooc.ooc_stats()
    rc = ooc.ooc_dgemm("N", "N", M, N, 0, 1.0, A, 1, B, N, -2.0, C, N, 1 << 20, None, st)
    assert rc == 0, ooc.ooc_last_error()
    assert np.array_equal(np64(C), -2.0 * C0)


def test_paper_mode_worked_example(ooc):
    A = pinned_from(7, 0, 4, 8, synth.INTEGER, 9)
    B = pinned_from(7, 1, 8, 4, synth.INTEGER, 9)
    C = pinned_from(7, 2, 4, 4, synth.INTEGER, 9)
    C0 = np64(C)
    opts = ooc.make_opts(flags=ooc.OOC_PLAN_PAPER)
    rc, st = run_dgemm(ooc, "N", "N", A, B, C, 1.0, 1.0, 44 * 8, opts)
    assert rc == 0, ooc.ooc_last_error()
    assert st.blocks == 8 and (st.mb, st.nb) == (1, 2)
    assert np.array_equal(np64(C), oracle.gemm("N", "N", 1.0, np64(A), np64(B), 1.0, C0))


def test_unpinned_host_memory_is_rejected(ooc):
    A = np.ones((16, 16))
    B = np.ones((16, 16))
    C = np.zeros((16, 16))
    rc = ooc.ooc_dgemm("N", "N", 16, 16, 16, 1.0, A, 16, B, 16, 0.0, C, 16, 1 << 20)
    assert rc == ooc.OOC_ERR_NOT_PINNED


@pytest.mark.parametrize("spec,code", [("alloc", -9), ("copy:3", -9), ("kernel:2", -9)])
def test_injected_failures_leave_library_usable(ooc, spec, code, monkeypatch):
    M, N, K = 200, 200, 200
    A = pinned_from(8, 0, M, K, synth.UNIFORM)
    B = pinned_from(8, 1, K, N, synth.UNIFORM)
    C = pinned(M, N, fill=0.0)
    opts = ooc.make_opts(mb=64, nb=64, kb=64)
    monkeypatch.setenv("OOC_FAULT_INJECT", spec)
    rc, _ = run_dgemm(ooc, "N", "N", A, B, C, 1.0, 0.0, 1 << 30, opts)
    assert rc == code
    monkeypatch.delenv("OOC_FAULT_INJECT")
    rc, _ = run_dgemm(ooc, "N", "N", A, B, C, 1.0, 0.0, 1 << 30, opts)
    assert rc == 0
    assert oracle.rel_fro(np64(C), oracle.gemm("N", "N", 1.0, np64(A), np64(B), 0.0, None)) <= TOL


def test_caller_workspace(ooc):
    M, N, K = 512, 384, 256
    A = pinned_from(9, 0, M, K, synth.NORMAL)
    B = pinned_from(9, 1, K, N, synth.NORMAL)
    C = pinned_from(9, 2, M, N, synth.NORMAL)
    C0 = np64(C)
    budget = 2 << 20
    ws = torch.empty(budget, dtype=torch.uint8, device="cuda")
    opts = ooc.make_opts(workspace=ws.data_ptr(), workspace_bytes=budget)
    rc, st = run_dgemm(ooc, "N", "N", A, B, C, 1.0, 1.0, budget, opts)
    assert rc == 0, ooc.ooc_last_error()
    assert oracle.rel_fro(np64(C), oracle.gemm("N", "N", 1.0, np64(A), np64(B), 1.0, C0)) <= TOL


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_device_entry_in_core(ooc, ta, tb):
    M, N, K = 333, 130, 257
    sa = (M, K) if ta == "N" else (K, M)
    sb = (K, N) if tb == "N" else (N, K)
    A = synth.matrix(*sa, 10, 0, synth.NORMAL)
    B = synth.matrix(*sb, 10, 1, synth.NORMAL)
    C = synth.matrix(M, N, 10, 2, synth.NORMAL)
    # even leading dimensions (TMA row pitch)
    dA = torch.zeros((sa[0], sa[1] + (sa[1] % 2)), dtype=torch.float64, device="cuda")
    dB = torch.zeros((sb[0], sb[1] + (sb[1] % 2)), dtype=torch.float64, device="cuda")
    dC = torch.zeros((M, N + (N % 2)), dtype=torch.float64, device="cuda")
    dA[:, :sa[1]] = torch.from_numpy(A)
    dB[:, :sb[1]] = torch.from_numpy(B)
    dC[:, :N] = torch.from_numpy(C)
    torch.cuda.synchronize()
    rc = ooc.ooc_dgemm_device(ta, tb, M, N, K, 0.75, dA, dA.stride(0), dB, dB.stride(0), -1.25, dC,
                              dC.stride(0), None)
    assert rc == 0, ooc.ooc_last_error()
    torch.cuda.synchronize()
    ref = oracle.gemm(ta, tb, 0.75, A, B, -1.25, C)
    assert oracle.rel_fro(dC[:, :N].cpu().numpy(), ref) <= TOL


def test_device_entry_clears_error_word_between_calls(ooc, monkeypatch):
    """ooc_dgemm_device keeps one error word per device and clears it on the caller's stream
    before each launch: a word left nonzero by an earlier call (injected on the host after the
    first call's kernel, as a wait that gave up would leave it) must not cut the next call's
    kernel short.  K spans many stages so the producer's waits take their slow path, which is
    where the word is read."""
    M, N, K = 512, 384, 4096
    A = synth.matrix(M, K, 11, 0, synth.NORMAL)
    B = synth.matrix(K, N, 11, 1, synth.NORMAL)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    ref = oracle.gemm("N", "N", 1.0, A, B, 0.0, np.zeros((M, N)))
    monkeypatch.setenv("OOC_FAULT_INJECT", "devword")
    for _ in range(2):
        dC = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
        rc = ooc.ooc_dgemm_device("N", "N", M, N, K, 1.0, dA, K, dB, N, 0.0, dC, N, None)
        assert rc == 0, ooc.ooc_last_error()
        torch.cuda.synchronize()
        assert oracle.rel_fro(dC.cpu().numpy(), ref) <= TOL
    monkeypatch.delenv("OOC_FAULT_INJECT")
    dC = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
    assert ooc.ooc_dgemm_device("N", "N", M, N, K, 1.0, dA, K, dB, N, 0.0, dC, N, None) == 0
    torch.cuda.synchronize()
    assert oracle.rel_fro(dC.cpu().numpy(), ref) <= TOL
