"""Writes paper_tmatrix.txt: the coefficient-rotation matrices printed in
Sec. 3 ("Example n = 3" and "Example n = 3, revisited"), evaluated at a few
angles.  The entries below are transcribed from the paper's two printed
matrices; nothing here calls the oracle or the CUDA path.

Rotating a filter by Theta maps its coefficient vector a to T(Theta) a.
  diagonal basis (e^{2i theta}, e^{-2i theta}, 1):
      T = diag(e^{-2i Theta}, e^{2i Theta}, 1)
  cos/sin basis (cos^2 theta, sin^2 theta, cos theta sin theta):
      T = [[cos^2, sin^2, -cos sin],
           [sin^2, cos^2,  cos sin],
           [sin 2Theta, -sin 2Theta, cos 2Theta]]
"""
import cmath
import math
import pathlib

ANGLES = [0.0, math.pi / 6, math.pi / 4, 1.0, 2.5, -0.7]


def diag_matrix(t):
    return [[cmath.exp(-2j * t), 0, 0], [0, cmath.exp(2j * t), 0], [0, 0, 1]]


def cossin_matrix(t):
    c, s = math.cos(t), math.sin(t)
    return [[c * c, s * s, -c * s],
            [s * s, c * c, c * s],
            [math.sin(2 * t), -math.sin(2 * t), math.cos(2 * t)]]


def main():
    lines = ["# Sec. 3 worked examples: coefficient rotation matrices T(Theta).",
             "# basis theta re(T00) im(T00) re(T01) im(T01) ... (row-major, 9 complex entries)"]
    for name, fn in (("diag", diag_matrix), ("cossin", cossin_matrix)):
        for t in ANGLES:
            m = fn(t)
            vals = []
            for row in m:
                for v in row:
                    v = complex(v)
                    vals += [f"{v.real:.17g}", f"{v.imag:.17g}"]
            lines.append(" ".join([name, f"{t:.17g}"] + vals))
    path = pathlib.Path(__file__).with_name("paper_tmatrix.txt")
    path.write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
