"""Reader of the text fixtures in this folder: '#' lines are comments (the
citations), '[name]' starts a block, every other line is whitespace-separated
numbers appended to the current block."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    blocks, cur = {}, None
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                blocks[cur] = []
                continue
            blocks[cur].append([float(t) for t in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}
