"""Mixed-radix transform plans on the host (no GPU): the radix sequences
make_radix_plan gives every power-of-two and even 7-smooth length up to 1024
(products, radix set, stage count, the even first / last radix the pruned
zero-padded halves need), the Stockham stage indexing of the kernels run
with those radices in numpy against numpy.fft, the twiddle-table length
(lcm of the padded edges), and the box edges the library takes."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
# mixed-radix edges whose three-component tile needs more than 256 threads
# (include/dda.h, dda_plan_create)
REJECTED = {210, 250, 270, 294, 350, 360, 378, 384, 392, 400, 420, 432, 448, 450, 480, 486, 490,
            500, 504}


def _smooth(v):
    for f in (2, 3, 5, 7):
        while v % f == 0:
            v //= f
    return v == 1


@pytest.fixture(scope="module")
def native(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("radix") / "radix_plan_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "native", "radix_plan_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    plans, tws = {}, {}
    for ln in out.splitlines():
        f = ln.split()
        if f[0] == "plan":
            L, pow2, hin, hout, nst = map(int, f[1:6])
            plans[L] = (bool(pow2), bool(hin), bool(hout), [int(r) for r in f[6:6 + nst]])
        else:
            tws[tuple(map(int, f[1:4]))] = int(f[4])
    return plans, tws


def test_plans_cover_every_length(native):
    plans, _ = native
    want = [L for L in range(2, 1025) if (L & (L - 1)) == 0 or (L % 2 == 0 and _smooth(L))]
    assert sorted(plans) == want
    for L, (pow2, hin, hout, r) in plans.items():
        assert math.prod(r) == L, L
        if pow2:
            assert len(r) <= 4 and all(x in (2, 4, 8, 16) for x in r) and hin and hout
        else:
            assert 2 <= len(r) <= 8 and all(x in (2, 3, 4, 5, 7) for x in r), (L, r)
            assert hin == (r[0] % 2 == 0) and hin, (L, r)
            if hout:
                assert r[-1] % 2 == 0, (L, r)
            # the power of two 2^a becomes one radix 2 (a odd) and radix-4 stages, so
            # there is an even last stage (pruned output half) from a = 3 on
            v2 = (L & -L).bit_length() - 1
            assert hout == (v2 >= 3), (L, r)


def _stockham(x, radices, inverse=False, half_in=False, half_out=False):
    """The kernels' stage indexing (smem_stage / smem_stage_mr): butterfly jb
    reads x[jb + q L/R], multiplies by w_L^(q k L/(Ns R)), k = jb mod Ns, takes
    an R-point DFT and writes y[(jb - k) R + k + q Ns]."""
    L = len(x)
    s = np.array(x, dtype=complex)
    sgn = 1.0 if inverse else -1.0
    Ns = 1
    for st, R in enumerate(radices):
        LR = L // R
        jb = np.arange(LR)
        k = jb % Ns
        q = np.arange(R)
        v = s[jb[:, None] + q[None, :] * LR]
        if half_in and st == 0:
            v[:, R // 2:] = 0.0  # the upper input half is never read
        v = v * np.exp(sgn * 2j * np.pi * (q[None, :] * k[:, None] * (L // (Ns * R))) / L)
        F = np.exp(sgn * 2j * np.pi * np.outer(q, q) / R)
        y = v @ F.T
        out = np.empty(L, dtype=complex)
        out[((jb - k) * R + k)[:, None] + q[None, :] * Ns] = y
        s = out
        Ns *= R
    return s


def test_stage_indexing_matches_numpy_fft(native):
    plans, _ = native
    rng = np.random.default_rng(7)
    for L, (pow2, hin, hout, r) in plans.items():
        if pow2 and L > 64:
            continue
        x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
        ref = np.fft.fft(x)
        assert np.abs(_stockham(x, r) - ref).max() <= 1e-12 * np.abs(ref).max() * L, L
        assert np.abs(_stockham(x, r, inverse=True) - np.fft.ifft(x) * L).max() <= \
            1e-12 * np.abs(ref).max() * L, L
        if hin:
            xh = x.copy()
            xh[L // 2:] = 0.0
            got = _stockham(np.concatenate([x[:L // 2], np.full(L - L // 2, np.nan)]), r,
                            half_in=True)
            assert np.abs(got - np.fft.fft(xh)).max() <= 1e-12 * np.abs(ref).max() * L, L


def test_twiddle_length_is_the_lcm(native):
    _, tws = native
    for (l, m, n), t in tws.items():
        assert t == math.lcm(2 * l, 2 * m, 2 * n), (l, m, n, t)


def test_box_edges_the_library_takes():
    from paper_1903_09802_gb300 import dda
    for e in range(2, 513, 2):
        ok = (e & (e - 1)) == 0 or (_smooth(e) and e not in REJECTED)
        got = dda.workspace_size(8, e, 8, 0.25, 2.0) > 0
        assert got == ok, e
    for e in (3, 9, 11, 13, 22, 26, 1024):
        assert dda.workspace_size(8, e, 8, 0.25, 2.0) == 0, e
