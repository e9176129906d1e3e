"""Reader for the hand-derived fixtures under tests/golden/."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_tree(name: str) -> dict:
    perm, clusters, blocks = None, [], []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "perm":
                perm = [int(x) for x in line[1:]]
            elif line[0] == "cluster":
                clusters.append(tuple(int(x) for x in line[1:]))
            elif line[0] == "block":
                blocks.append(tuple(int(x) for x in line[1:]))
    return dict(perm=perm, clusters=clusters, blocks=blocks)


def tree_hash(nodes: dict) -> str:
    """SHA-256 of a block tree's (row cluster, column cluster, kind) node
    arrays in pre-order, as little-endian int32 (the key the stored oracle
    values of tests/golden/oracle_*.json carry)."""
    import hashlib

    import numpy as np
    h = hashlib.sha256()
    for key in ("t", "s", "kind"):
        h.update(np.ascontiguousarray(nodes[key], dtype="<i4").tobytes())
    return h.hexdigest()


def perm_hash(perm) -> str:
    import hashlib

    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(perm, dtype="<i8").tobytes()).hexdigest()


def read_oracle_values(workload: str):
    """The oracle's stored values for a full-size workload, or None."""
    import json
    path = os.path.join(HERE, f"oracle_{workload}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)
