"""Loader for the text fixtures in tests/golden (``key = numbers`` lines, ``#`` comments)."""
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(_HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            nums = [float(t) for t in val.split()]
            out[key] = int(nums[0]) if len(nums) == 1 and float(nums[0]).is_integer() else np.array(nums)
    return out
