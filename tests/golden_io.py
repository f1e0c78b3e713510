"""Reader for the hand-worked fixtures in tests/golden/."""
from __future__ import annotations

import os
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = line.split(":", 1)
            out[key.strip()] = val.strip()
    return out


def fractions(text: str):
    return [Fraction(tok) for tok in text.split()]


def ints(text: str):
    return [int(tok) for tok in text.split()]
