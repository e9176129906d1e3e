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
