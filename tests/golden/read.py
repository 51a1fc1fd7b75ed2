"""Readers of the text fixtures in this folder (values printed in the paper, each row
with its citation)."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(name):
    with open(os.path.join(_HERE, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def paper_fmm_errors():
    """{case: (E_V, E_delta)} as fractions (the fixture holds percent)."""
    return {r[0]: (float(r[1]) / 100.0, float(r[2]) / 100.0) for r in _rows("paper_fmm_errors.txt")}


def paper_kernel_coeffs():
    """{model: [(coefficient, lambda), ...]} in the table's row order."""
    out = {}
    for r in _rows("paper_kernel_coeffs.txt"):
        out.setdefault(r[0], []).append((float(r[2]), float(r[3])))
    return out


def paper_constants():
    return {r[0]: float(r[1]) for r in _rows("paper_constants.txt")}
