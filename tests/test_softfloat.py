"""libssa's integer FP64 routines (csrc/ssa_softfloat.cuh), compiled for the
host, against the CPU's IEEE round-to-nearest-even double arithmetic:
products c * h (h < 2^53), quotients, integer-to-double conversions,
power-of-two scaling and (exhaustively) binary32-to-binary64 widening, with edge significands (all zeros, all ones, one ulp).
The same source is compiled for the GPU; the GPU parity tests then check the
whole step bit for bit."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_softfloat_matches_ieee():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "sfcheck")
        subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-Wno-unknown-pragmas",
                        "-I", os.path.join(ROOT, "paper_1007_1768_gb300", "csrc"), "-o", exe,
                        os.path.join(ROOT, "tests", "softfloat_check.cpp")], check=True)
        for seed in (1, 2):
            r = subprocess.run([exe, "2000000", str(seed)], capture_output=True, text=True)
            lines = {l.split()[0]: [int(v) for v in l.split()[1:]] for l in r.stdout.splitlines()
                     if l.split() and l.split()[0] in ("mul", "div", "cvt", "scale", "widen")}
            assert r.returncode == 0, r.stdout
            for op in ("mul", "div", "cvt", "scale"):
                tested, bad, _ = lines[op]
                assert tested == 2000000 and bad == 0, (op, lines[op])
            tested, bad, _ = lines["widen"]
            assert tested == 0x7F800001 and bad == 0, lines["widen"]
