"""Slips planted in a copy of the oracle are caught by its pins (CPU only).

Each case below changes one expression of oracle/lacos_oracle.cpp the way a
plausible mistake would -- a dropped term, a wrong sign, index, window or
threshold, a missing exclusion -- compiles the changed copy, and runs the
oracle's pin tests (tests/test_oracle_pins.py, tests/test_oracle_gain.py)
against it in a child process through LACOS_ORACLE_LIB.  The pins must fail
for every slip; the unchanged copy, built the same way, must pass them.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lacos_oracle.cpp")
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_gain.py")]

pytestmark = pytest.mark.slow

# (name, exact text in the oracle source, its replacement)
SLIPS = [
    ("laplacian term dropped", "const T c4 = std::max(T(0), (vv - d) - r);", "const T c4 = T(0);"),
    ("S over N instead of 2N", "S[q] = L[q] / (N[q] + N[q]);", "S[q] = L[q] / N[q];"),
    ("read noise not squared", "const T rn2 = p.readnoise * p.readnoise;", "const T rn2 = p.readnoise;"),
    ("noise floor dropped", "const T e = std::max(g * m5[q], T(1e-4));", "const T e = g * m5[q];"),
    ("sign of S'", "Sp[q] = S[q] - mS[q];", "Sp[q] = mS[q] - S[q];"),
    ("F not divided by N", "F[q] = p.fnorm ? std::max(diff / N[q], T(0.01))", "F[q] = p.fnorm ? std::max(diff, T(0.01))"),
    ("med7 window taken as 5x5", "median_filter(m3.data(), ny, nx, 7, m7.data());",
     "median_filter(m3.data(), ny, nx, 5, m7.data());"),
    ("med3 window taken as 5x5", "median_filter(I, ny, nx, 3, m3.data());", "median_filter(I, ny, nx, 5, m3.data());"),
    ("objlim numerator S instead of S'", "(Sp[q] / F[q]) > p.objlim", "(S[q] / F[q]) > p.objlim"),
    ("candidates without the saturation test", "cand[q] = (!sat[q] && Sp[q] > p.sigclip", "cand[q] = (Sp[q] > p.sigclip"),
    ("first growth re-tested at sigfrac*sigclip", "g1[q] = (d1[q] && Sp[q] > p.sigclip && !sat[q])",
     "g1[q] = (d1[q] && Sp[q] > p.sigfrac * p.sigclip && !sat[q])"),
    ("lower growth threshold taken as sigclip", "const T lo = p.sigfrac * p.sigclip;", "const T lo = p.sigclip;"),
    ("non-strict threshold", "g2[q] = (d2[q] && Sp[q] > lo && !sat[q])", "g2[q] = (d2[q] && Sp[q] >= lo && !sat[q])"),
    ("dilation without the left neighbours", "for (int dj = -1; dj <= 1; ++dj) {\n          const int y = i + di, x = j + dj;",
     "for (int dj = 0; dj <= 1; ++dj) {\n          const int y = i + di, x = j + dj;"),
    ("upper median in the replacement", "*out = pool[(pool.size() - 1) / 2];", "*out = pool[pool.size() / 2];"),
    ("replacement pool includes flagged pixels", "if (!M[q]) pool.push_back(X0[q]);", "pool.push_back(X0[q]);"),
    ("median window not clamped at the border",
     "w[n++] = A[(size_t)clampi(i + di, 0, ny - 1) * nx + clampi(j + dj, 0, nx - 1)];",
     "if (i + di >= 0 && i + di < ny && j + dj >= 0 && j + dj < nx) w[n++] = A[(size_t)(i + di) * nx + (j + dj)];"),
    ("no early stop", "if (fresh == 0) break;", "(void)fresh;"),
    ("gain: read-noise term dropped", "const double disc = A * A + 8.0 * nd * rn2 * V;", "const double disc = A * A;"),
    ("gain: 2-sigma clip", "const __int128 bound = 9 * (n * s2 - s1 * s1);", "const __int128 bound = 4 * (n * s2 - s1 * s1);"),
    ("gain: sample variance", "const double V = (double)vnum / nd;", "const double V = (double)vnum / (nd - 1.0);"),
    ("gain: flagged partner kept", "if (M[q] || M[q + 1] || sat[q] || sat[q + 1]) continue;",
     "if (M[q] || sat[q] || sat[q + 1]) continue;"),
    ("gain: three clipping rounds", "if (st.n == 0 || r == 5 || (r > 0 && st.n == prev.n)) break;",
     "if (st.n == 0 || r == 3 || (r > 0 && st.n == prev.n)) break;"),
]


def _build(src_text, out):
    cpp = out + ".cpp"
    with open(cpp, "w") as f:
        f.write(src_text)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    cpp, "-o", out], check=True)
    return out


def _pins(lib):
    env = dict(os.environ, LACOS_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def outcomes(source, tmp_path_factory):
    """Every copy (the unchanged one first) built and run against the pins, several at a
    time (each is a compiler and a pytest process of its own)."""
    from concurrent.futures import ThreadPoolExecutor
    d = tmp_path_factory.mktemp("slips")
    texts = [("unchanged", source)] + [(name, source.replace(old, new)) for name, old, new in SLIPS]

    def one(i_text):
        i, (name, text) = i_text
        return name, _pins(_build(text, str(d / f"copy{i}.so")))

    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(one, enumerate(texts)))


def test_unchanged_copy_passes_the_pins(outcomes):
    rc, out = outcomes["unchanged"]
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new", SLIPS, ids=[s[0] for s in SLIPS])
def test_planted_slip_is_caught(source, outcomes, name, old, new):
    assert source.count(old) == 1, f"the text of '{name}' no longer occurs once in the oracle"
    rc, out = outcomes[name]
    assert rc != 0 and "failed" in out, f"slip not caught: {name}\n{out}"
