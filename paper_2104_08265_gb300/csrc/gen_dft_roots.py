"""Writes dft_roots.cuh: cos and sin of 2 pi m / R rounded to float, for the register DFT
radices of the FFT engine.  Run: python gen_dft_roots.py (output next to this file)."""
import math
import os
import struct

RADICES = [6, 9, 10, 12, 14, 15, 18, 20, 24, 25, 27, 28, 30, 32]


def f32(x: float) -> str:
    v = struct.unpack("f", struct.pack("f", x))[0]
    s = repr(v)
    if "e" not in s and "." not in s:
        s += ".0"
    return s + "f"


def cos_sin(m: int, R: int):
    """cos, sin (2 pi m / R), exact at multiples of a quarter turn."""
    if (4 * m) % R == 0:
        return [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)][(4 * m) // R]
    a = 2 * math.pi * m / R
    return math.cos(a), math.sin(a)


def main():
    out = ["// Generated by gen_dft_roots.py: cos / sin (2 pi m / R) rounded to float.",
           "#pragma once", "", "namespace wcsim {", "",
           "template <int R> struct Roots;", ""]
    for R in RADICES:
        c = ", ".join(f32(cos_sin(m, R)[0]) for m in range(R))
        s = ", ".join(f32(cos_sin(m, R)[1]) for m in range(R))
        out += ["template <> struct Roots<%d> {" % R,
                "    static __host__ __device__ constexpr float c(int m) { constexpr float t[%d] = {%s}; return t[m]; }" % (R, c),
                "    static __host__ __device__ constexpr float s(int m) { constexpr float t[%d] = {%s}; return t[m]; }" % (R, s),
                "};", ""]
    out += ["}  // namespace wcsim", ""]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dft_roots.cuh")
    open(path, "w").write("\n".join(out))
    print(path)


if __name__ == "__main__":
    main()
