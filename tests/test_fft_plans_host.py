"""The library's FFT stages (csrc/fft_core.cuh: the radix codelets, the
mixed-radix decimation-in-frequency stages, the digit-reversed output order
and the transposed inverse stages), compiled for the host in double and run
on every plan the pair and orbital transforms use -- make_axis_plan's for each
compile-time cube and other 2-3-5 lengths, and the two-stage alternatives the
autotuner times -- against numpy's FFT: the forward transform read through
digit_reversed_position, and the inverse stages taking that digit-reversed
spectrum back to n times the input in natural order."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2110_07670_gb300", "csrc")
DRIVER = r"""
#include <cstdio>
#include <cmath>
#include <vector>
#include "fft_core.cuh"
using namespace ace;
template <int SGN>
void run_stage(int r, std::vector<cx<double>>& buf, const Lines& L, const cx<double>* tw, int Lb) {
    const int nb = L.n / r;
    for (int b = 0; b < nb * L.nlines; ++b) {
        switch (r) {
            case 2: stage_butterfly<2, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 3: stage_butterfly<3, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 4: stage_butterfly<4, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 5: stage_butterfly<5, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 6: stage_butterfly<6, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 8: stage_butterfly<8, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 9: stage_butterfly<9, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 10: stage_butterfly<10, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 12: stage_butterfly<12, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 15: stage_butterfly<15, SGN, double>(buf.data(), L, tw, Lb, b); break;
            case 16: stage_butterfly<16, SGN, double>(buf.data(), L, tw, Lb, b); break;
        }
    }
}
int main() {
    int n, r0;
    while (std::scanf("%d %d", &n, &r0) == 2) {
        AxisPlan P{};
        bool ok = r0 ? make_axis_plan_first(n, r0, P) : make_axis_plan(n, P);
        std::printf("plan %d %d %d", n, r0, ok ? P.nstages : -1);
        for (int s = 0; s < P.nstages; ++s) std::printf(" %d", P.radix[s]);
        std::printf("\n");
        std::vector<cx<double>> x(n), tw(n);
        for (int k = 0; k < n; ++k) { double a = -2 * M_PI * k / n; tw[k] = mk(std::cos(a), std::sin(a)); }
        for (int k = 0; k < n; ++k)
            if (std::scanf("%lf %lf", &x[k].re, &x[k].im) != 2) return 1;
        if (!ok) continue;
        Lines L{n, 1, 1, n};
        std::vector<cx<double>> f = x;
        int Lb = n;
        for (int s = 0; s < P.nstages; ++s) { run_stage<-1>(P.radix[s], f, L, tw.data(), Lb); Lb /= P.radix[s]; }
        for (int k = 0; k < n; ++k) { const cx<double> v = f[digit_reversed_position(P, k)]; std::printf("%.17g %.17g\n", v.re, v.im); }
        std::vector<cx<double>> g = f;  // inverse of the digit-reversed spectrum
        Lb = 1;
        for (int s = P.nstages - 1; s >= 0; --s) { Lb *= P.radix[s]; run_stage<+1>(P.radix[s], g, L, tw.data(), Lb); }
        for (int k = 0; k < n; ++k) std::printf("%.17g %.17g\n", g[k].re, g[k].im);
    }
}

"""

CASES = [(n, 0) for n in (2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48, 50, 54,
                          60, 64, 72, 75, 80, 81, 90, 96, 100, 108, 120, 125, 128, 144, 150, 160, 180, 200, 240)] + \
        [(96, 8), (96, 16), (120, 10), (120, 8), (160, 10)]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("fft")
    src = d / "fft_host.cpp"
    src.write_text(DRIVER)
    exe = d / "fft_host"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def test_fft_stages_against_numpy(driver):
    rng = np.random.default_rng(2110)
    inputs = {case: rng.standard_normal(case[0]) + 1j * rng.standard_normal(case[0]) for case in CASES}
    text = "".join(f"{n} {r0}\n" + "".join(f"{float(v.real)!r} {float(v.imag)!r}\n" for v in inputs[(n, r0)])
                   for n, r0 in CASES)
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    pos = 0
    for n, r0 in CASES:
        head = out[pos].split()
        pos += 1
        assert head[:3] == ["plan", str(n), str(r0)] and int(head[3]) >= 1, head
        radices = [int(r) for r in head[4:]]
        assert int(np.prod(radices)) == n
        if r0:
            assert radices == [r0, n // r0]
        vals = np.array([complex(*map(float, out[pos + k].split())) for k in range(2 * n)])
        pos += 2 * n
        x = inputs[(n, r0)]
        scale = np.abs(x).sum()
        assert np.abs(vals[:n] - np.fft.fft(x)).max() <= 1e-13 * scale, (n, r0)
        assert np.abs(vals[n:] - n * x).max() <= 1e-13 * n * scale, (n, r0)
