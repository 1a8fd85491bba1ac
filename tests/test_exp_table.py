"""The exponential's constants and tables (csrc/exp_table.inc) are what the
committed generator (csrc/gen_exp_table.py, 50-digit decimal arithmetic
from their definitions) writes, and they satisfy those definitions:
T_hi[j] + T_lo[j] = 2^(j/256) to about 2^-105, L1 + L2 = ln 2 / 256 (to half
an ulp of L2) with N L1 exact for N < 2^21, the integer form of L1, and the FP32 pieces of the
float-float polynomial (T_hi = TH + TL with TH its leading 24 bits, TL and
T_lo rounded to FP32)."""
import math
import os
import re
import struct
import subprocess
import sys
from decimal import Decimal, getcontext


CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2607_23354_gb300", "csrc")


def _inc():
    with open(os.path.join(CSRC, "exp_table.inc")) as f:
        return f.read()


def test_generator_reproduces_the_committed_table():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp_table.py")], capture_output=True, text=True,
                         check=True).stdout
    assert out == _inc()


def _define(txt, name):
    m = re.search(r"#define %s (\S+)" % name, txt)
    return m.group(1)


def _f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def test_table_entries_match_their_definitions():
    getcontext().prec = 50
    txt = _inc()
    body = txt[txt.index("kExpTable[512]"):txt.index("};")]
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == 512
    for j in range(256):
        exact = Decimal(2) ** (Decimal(j) / Decimal(256))
        hi, lo = vals[2 * j], vals[2 * j + 1]
        assert abs(Decimal(hi) + Decimal(lo) - exact) <= Decimal(2) ** -104 * exact
        assert abs(lo) <= math.ulp(hi)
    l1 = float.fromhex(_define(txt, "EXPT_L1"))
    l2 = float.fromhex(_define(txt, "EXPT_L2"))
    ln2_256 = Decimal(2).ln() / Decimal(256)
    # L2 is the remainder rounded to a double: within half its unit in the last place
    assert abs(Decimal(l1) + Decimal(l2) - ln2_256) <= Decimal(math.ulp(l2)) / 2
    m, _ = math.frexp(l1)
    assert int(m * 2 ** 53) % (1 << 21) == 0  # N L1 exact for N < 2^21
    l1m = int(_define(txt, "EXPT_L1M").rstrip("ul"), 16)
    l1e = int(_define(txt, "EXPT_L1E").strip("()"))
    assert l1m * 2.0 ** l1e == l1 and l1m < 2 ** 32
    # the FP32 pieces: 16-byte entries (T_hi low word, high word, TL, T_lo)
    xbody = txt[txt.index("kExpTableX"):]
    words = [int(w, 16) for w in re.findall(r"0x([0-9a-f]{8})u", xbody)]
    assert len(words) == 1024
    for j in range(256):
        lo32, hi32, tlb, tlob = words[4 * j:4 * j + 4]
        th = struct.unpack("<d", struct.pack("<Q", (hi32 << 32) | lo32))[0]
        assert th == vals[2 * j]
        lead = struct.unpack("<d", struct.pack("<Q", ((hi32 << 32) | lo32) & ~((1 << 29) - 1)))[0]
        tl = struct.unpack("<f", struct.pack("<I", tlb))[0]
        assert tl == _f32(th - lead)
        assert struct.unpack("<f", struct.pack("<I", tlob))[0] == _f32(vals[2 * j + 1])
    for name, value in (("EXPT_L2", l2), ("S6", 1.0 / 6.0)):
        if name == "S6":
            h = float.fromhex(_define(txt, "EXPT_S6H").rstrip("f"))
            lo = float.fromhex(_define(txt, "EXPT_S6L").rstrip("f"))
            exact = Decimal(1) / Decimal(6)
        else:
            h = float.fromhex(_define(txt, "EXPT_L2H").rstrip("f"))
            lo = float.fromhex(_define(txt, "EXPT_L2L").rstrip("f"))
            exact = Decimal(value)
        assert h == _f32(h) and lo == _f32(lo)
        assert abs(Decimal(h) + Decimal(lo) - exact) <= Decimal(2) ** -46 * abs(exact)
