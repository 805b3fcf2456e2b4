"""The band save/restore kernels index a band region by two divisions, done
as a multiply-high and a shift with multipliers that the host computes once
per region (`band_divisor` in csrc/smi_internal.h, after Granlund and
Montgomery 1994).  This CPU test compiles that host function with g++ and
checks (mulhi(m, u) + u) >> l == u / d against exact division for every
divisor up to 4096, for large divisors, and for u across [0, 2^31) including
the ends of each quotient interval."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include <cstdint>
#include "smi_internal.h"
static unsigned mulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
static unsigned long long rng = 88172645463325252ull;
static unsigned next() { rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17; return (unsigned)(rng >> 33); }
int main() {
    long long bad = 0, checked = 0;
    auto check = [&](unsigned d, unsigned u) {
        unsigned m; int l;
        smi::band_divisor(d, m, l);
        const unsigned q = (mulhi(m, u) + u) >> l;
        checked++;
        if (q != u / d) { if (bad < 5) std::printf("d=%u u=%u q=%u\n", d, u, q); bad++; }
    };
    for (unsigned d = 1; d <= 4096; d++) {
        const unsigned top = 0x7fffffffu;
        unsigned us[] = {0u, 1u, d - 1, d, d + 1, 2 * d - 1, 2 * d, top, top - 1, top / d * d, top / d * d - 1};
        for (unsigned u : us) if (u <= top) check(d, u);
        for (int k = 0; k < 200; k++) check(d, next() & 0x7fffffffu);
    }
    for (int k = 0; k < 2000; k++) {
        const unsigned d = 1 + (next() % 0x7fffffffu);
        for (int j = 0; j < 20; j++) check(d, next() & 0x7fffffffu);
        check(d, d); check(d, d - 1);
    }
    std::printf("checked %lld bad %lld\n", checked, bad);
    return bad != 0;
}
'''


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_band_divisor_equals_exact_division():
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "t.cpp")
        exe = os.path.join(tmp, "t")
        with open(src, "w") as f:
            f.write(SRC)
        inc = ["-I", os.path.join(ROOT, "paper_2311_02293_gb300", "csrc"), "-I", os.path.join(ROOT, "include")]
        subprocess.run(["g++", "-std=c++17", "-O2", *inc, src, "-o", exe], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout
        assert "bad 0" in r.stdout
