"""CPU checks of the GPU library's per-element math (compiled for the host from
the same headers the kernels use): harmonic recurrences, Stockham butterflies,
the real-matrix M2L of one wavevector, and L2P with the order-one gradient.
References: the FP64 oracle and numpy's FFT."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host", "host_math.cpp")
INC = os.path.join(ROOT, "paper_1409_5981_gb300", "csrc")
OUT = os.path.join(HERE, "_build", "libhostmath.so")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    deps = [SRC] + [os.path.join(INC, f) for f in ("common.cuh", "harmonics.cuh", "translations.cuh", "fft.cuh",
                                                   "m2l_table.cuh")]
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(d) for d in deps):
        tmp = OUT + f".{os.getpid()}"
        subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", INC, "-o", tmp, SRC], check=True)
        os.replace(tmp, OUT)
    L = ctypes.CDLL(OUT)
    vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    L.h_regular_real.argtypes = [i, d, d, d, vp]
    L.h_singular_real.argtypes = [i, d, d, d, vp]
    L.h_fft.argtypes = [i, i, i, vp]
    L.h_m2l_k.argtypes = [i, vp, vp, vp]
    L.h_m2l_k_par.argtypes = [i, vp, vp, vp]
    L.h_l2p.argtypes = [i, vp, vp, vp]
    L.h_m2l_table.argtypes = [i, vp, vp, vp]
    L.h_l2p_stream.argtypes = [i, vp, vp, vp]
    L.h_regular_stream.argtypes = [i, d, d, d, vp]
    return L


def P(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_regular_recurrence_vs_oracle(lib):
    g = synth.rng(101)
    for p in range(0, lib.h_pmax() + 1):
        for _ in range(5):
            r = g.standard_normal(3) * 0.7
            out = np.zeros((p + 1) ** 2)
            lib.h_regular_real(p, *r, P(out))
            ref = oracle.to_real_storage(oracle.solid_R(p, r))
            assert np.abs(out - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()), p


def test_singular_recurrence_vs_oracle(lib):
    g = synth.rng(102)
    for J in (0, 1, 4, 9, 16, 24):
        for _ in range(5):
            r = g.standard_normal(3) * 2.0
            out = np.zeros((J + 1) ** 2)
            lib.h_singular_real(J, *r, P(out))
            ref = oracle.to_real_storage(oracle.solid_S(J, r))
            for j in range(J + 1):
                sl = slice(j * j, (j + 1) ** 2)
                assert np.abs(out[sl] - ref[sl]).max() <= 1e-12 * np.abs(ref[sl]).max(), (J, j)


@pytest.mark.parametrize("single", [0, 1])
def test_stockham_vs_numpy(lib, single):
    g = synth.rng(103)
    for logL in range(1, 10):
        L = 1 << logL
        x = g.standard_normal(L) + 1j * g.standard_normal(L)
        for inv in (0, 1):
            buf = np.ascontiguousarray(np.stack([x.real, x.imag], -1).reshape(-1))
            lib.h_fft(L, inv, single, P(buf))
            y = buf[0::2] + 1j * buf[1::2]
            ref = np.fft.ifft(x) * L if inv else np.fft.fft(x)
            tol = (2e-6 if single else 1e-13) * np.abs(ref).max() * logL
            assert np.abs(y - ref).max() < tol, (L, inv)


def _hermitian_real_storage(p, g):
    """Random complex harmonics obeying X_l^{-m} = (-1)^m conj X_l^m, and their real storage."""
    X = g.standard_normal((p + 1) ** 2) + 1j * g.standard_normal((p + 1) ** 2)
    for l in range(p + 1):
        X[oracle.hidx(l, 0)] = X[oracle.hidx(l, 0)].real
        for m in range(1, l + 1):
            X[oracle.hidx(l, -m)] = (-1) ** m * np.conj(X[oracle.hidx(l, m)])
    return X, oracle.to_real_storage(X)


def test_real_matrix_m2l_vs_complex_form(lib):
    """App. A.8: the real-matrix M2L equals the complex Eq. M2L on real storage."""
    g = synth.rng(104)
    for p in (0, 1, 2, 4, 7, 10, 12):
        M, Mr = _hermitian_real_storage(p, g)
        d = g.standard_normal(3) + np.array([3.0, 0, 0])
        S = oracle.solid_S(2 * p, d)
        Sr = oracle.to_real_storage(S)
        Lref = oracle.to_real_storage(oracle.m2l_green(p, M, S))
        Mc = np.stack([Mr, np.zeros_like(Mr)], -1).reshape(-1).copy()
        Gc = np.stack([Sr, np.zeros_like(Sr)], -1).reshape(-1).copy()
        Lc = np.zeros(2 * (p + 1) ** 2)
        lib.h_m2l_k(p, P(Mc), P(Gc), P(Lc))
        assert np.abs(Lc[0::2] - Lref).max() < 1e-12 * np.abs(Lref).max(), p
        assert np.abs(Lc[1::2]).max() == 0.0


def test_real_matrix_m2l_in_fourier_space(lib):
    """Sec. 2.1: per-wavevector real-matrix M2L on the spectra of the real channels,
    then an inverse FFT, equals the cyclic cell sum L_i = sum_j G_{i-j} M_j (complex form)."""
    g = synth.rng(105)
    p, n = 3, 4
    C, CG = (p + 1) ** 2, (2 * p + 1) ** 2
    K = n ** 3
    Mc = np.zeros((K, C), dtype=complex)
    Mr = np.zeros((K, C))
    for i in range(K):
        Mc[i], Mr[i] = _hermitian_real_storage(p, g)
    Gc = np.zeros((K, CG), dtype=complex)
    Gr = np.zeros((K, CG))
    for i in range(K):
        Gc[i], Gr[i] = _hermitian_real_storage(2 * p, g)
    # reference: direct cyclic sum, complex form
    idx = np.array(np.unravel_index(np.arange(K), (n, n, n))).T
    Lref = np.zeros((K, C), dtype=complex)
    for i in range(K):
        for j in range(K):
            dd = tuple((idx[i] - idx[j]) % n)
            k = np.ravel_multi_index(dd, (n, n, n))
            Lref[i] = oracle.m2l_green(p, Mc[j], Gc[k], Lref[i])
    Lref_r = oracle.to_real_storage(Lref)
    # FFT path: per-channel full complex FFT of the real fields (numpy), per-k M2L, inverse
    Mt = np.fft.fftn(Mr.reshape(n, n, n, C), axes=(0, 1, 2)).reshape(K, C)
    Gt = np.fft.fftn(Gr.reshape(n, n, n, CG), axes=(0, 1, 2)).reshape(K, CG)
    Lt = np.zeros((K, C), dtype=complex)
    for k in range(K):
        mbuf = np.stack([Mt[k].real, Mt[k].imag], -1).reshape(-1).copy()
        gbuf = np.stack([Gt[k].real, Gt[k].imag], -1).reshape(-1).copy()
        lbuf = np.zeros(2 * C)
        lib.h_m2l_k(p, P(mbuf), P(gbuf), P(lbuf))
        Lt[k] = lbuf[0::2] + 1j * lbuf[1::2]
    L = np.fft.ifftn(Lt.reshape(n, n, n, C), axes=(0, 1, 2)).reshape(K, C)
    assert np.abs(L.imag).max() < 1e-10 * np.abs(Lref_r).max()
    assert np.abs(L.real - Lref_r).max() < 1e-11 * np.abs(Lref_r).max()


def test_l2p_real_form_vs_oracle(lib):
    g = synth.rng(106)
    for p in (0, 1, 2, 5, 9, 12):
        Lc, Lr = _hermitian_real_storage(p, g)
        u = g.random(3) - 0.5
        out = np.zeros(4)
        lib.h_l2p(p, P(np.ascontiguousarray(Lr)), P(np.ascontiguousarray(u)), P(out))
        phi, grad = oracle.l2p(p, Lc, u)
        assert abs(out[0] - phi) < 1e-12 * max(1, abs(phi))
        if p >= 1:
            assert np.abs(out[1:] - grad).max() < 1e-12 * max(1, np.abs(grad).max())


def test_streamed_harmonics_and_l2p_vs_oracle(lib):
    """Column-by-column harmonics equal the oracle's R_l^m; the streamed L2P (harmonics
    on the fly, two columns kept) equals the oracle's L2P and gradient."""
    g = synth.rng(108)
    for p in (0, 1, 2, 3, 7, 11, 12):
        for _ in range(3):
            r = g.standard_normal(3) * 0.6
            out = np.zeros((p + 1) ** 2)
            lib.h_regular_stream(p, *r, P(out))
            ref = oracle.to_real_storage(oracle.solid_R(p, r))
            assert np.abs(out - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()), p
            Lc, Lr = _hermitian_real_storage(p, g)
            u = g.random(3) - 0.5
            res = np.zeros(4)
            lib.h_l2p_stream(p, P(np.ascontiguousarray(Lr)), P(np.ascontiguousarray(u)), P(res))
            phi, grad = oracle.l2p(p, Lc, u)
            assert abs(res[0] - phi) < 1e-12 * max(1, abs(phi)), p
            if p >= 1:
                assert np.abs(res[1:] - grad).max() < 1e-12 * max(1, np.abs(grad).max()), p


def test_m2l_entry_table_matches_per_k_m2l(lib):
    """The batched M2L's explicit matrix (entry table of App. A.8's real form) equals the
    per-wavevector real-matrix M2L on complex (Fourier-space) inputs."""
    g = synth.rng(107)
    for p in (0, 1, 3, 7, 11):
        C, CG = (p + 1) ** 2, (2 * p + 1) ** 2
        M = np.ascontiguousarray(g.standard_normal(2 * C))
        G = np.ascontiguousarray(g.standard_normal(2 * CG))
        a = np.zeros(2 * C)
        b = np.zeros(2 * C)
        lib.h_m2l_k(p, P(M), P(G), P(a))
        lib.h_m2l_table(p, P(M), P(G), P(b))
        assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(a).max()), p


def test_parity_m2l_equals_complex_form(lib):
    """The M2L on parity-reduced kernel spectra (component s of order j: real spectrum
    for even j, imaginary for odd j, one real number stored) equals the real-matrix
    form on the full complex spectra with that structure, for every p."""
    g = synth.rng(107)
    for p in range(0, lib.h_pmax() + 1):
        C, CG = (p + 1) ** 2, (2 * p + 1) ** 2
        Mc = g.standard_normal(2 * C)
        Gr = g.standard_normal(CG)
        Gc = np.zeros(2 * CG)
        for s in range(CG):
            j = int(np.floor(np.sqrt(s)))
            Gc[2 * s + (j & 1)] = Gr[s]
        L1 = np.zeros(2 * C)
        L2 = np.zeros(2 * C)
        lib.h_m2l_k(p, P(Mc), P(Gc), P(L1))
        lib.h_m2l_k_par(p, P(Mc), P(Gr), P(L2))
        assert np.abs(L1 - L2).max() <= 1e-13 * max(1.0, np.abs(L1).max()), p
