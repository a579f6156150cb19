"""Parser for the hand-position fixtures in this folder."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def hand_positions():
    cases = []
    cur = None
    rows = None
    with open(os.path.join(HERE, "hand_positions.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("case "):
                cur = {"name": line[5:].strip(), "rows": [], "expect": []}
            elif line == "board":
                rows = cur["rows"]
            elif line.startswith("expect "):
                rows = None
                parts = line.split()
                beta = int(parts[1])
                kv = dict(p.split("=") for p in parts[2:])
                cur["expect"].append((beta, int(kv["win"]), int(kv["notlose"])))
            elif line == "end":
                cases.append(cur)
                cur = rows = None
            elif rows is not None:
                rows.append(line)
    for c in cases:
        assert len(c["rows"]) == 6 and all(len(r) == 6 for r in c["rows"]), c["name"]
        c["cells"] = [".XO".index(ch) for r in c["rows"] for ch in r]
    return cases
