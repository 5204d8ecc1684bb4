"""Parser for tests/golden/codec_stream_small.txt (hand-derived codec streams)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "codec_stream_small.txt")


def load_cases(path: str = GOLDEN):
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "case":
                cur = dict(name=rest[0], x=[], v=[], hex=b"", repeat=1)
            elif key in ("n_fine", "n_cmp", "vel_bits", "repeat"):
                cur[key] = int(rest[0])
            elif key == "x":
                cur["x"].append([float(t) for t in rest])
            elif key == "v":
                cur["v"].append([float(t) for t in rest])
            elif key == "hex":
                cur["hex"] += bytes.fromhex("".join(rest))
            elif key == "hexrepeat":
                cur["hex"] += bytes.fromhex("".join(rest[1:])) * int(rest[0])
            elif key == "end":
                x = np.array(cur["x"], np.float32)
                v = np.array(cur["v"], np.float32)
                if cur["repeat"] > 1:
                    x = np.repeat(x, cur["repeat"], axis=0)
                    v = np.repeat(v, cur["repeat"], axis=0)
                cur["x"], cur["v"] = x, v
                cases.append(cur)
                cur = None
    return cases
