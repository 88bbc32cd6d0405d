"""Readers for the text fixtures beside this file: values printed in the paper, each file citing
the table or equation it is taken from."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def table_i():
    """Table I (Section II.F) as {K_max: (kappa, alpha, (c_0, ..., c_K))}."""
    rows = {}
    with open(os.path.join(HERE, "table_i.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            kmax = int(line[0])
            c = tuple(int(x) for x in line[3:])
            if len(c) != kmax + 1:
                raise ValueError(f"Table I row K_max = {kmax} has {len(c)} coefficients")
            rows[kmax] = (float(line[1]), float(line[2]), c)
    return rows
