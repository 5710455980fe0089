"""Reads tests/golden/paper_values.txt (values printed in the paper)."""

import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_values.txt")


def paper_values():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out
