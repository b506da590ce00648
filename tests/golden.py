"""Loader of the paper's printed values under tests/golden/ (each file names
the table it comes from)."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def taylor_bubble_re():
    """{D: Re of the paper's PFLBM}, and the experiment's Re."""
    re, exp = {}, None
    for r in _rows("taylor_bubble_re.txt"):
        if r[0] == "experiment":
            exp = float(r[1])
        else:
            re[int(r[0])] = float(r[1])
    return re, exp


def drop_table(case):
    """case 'vertical' or 'oblique' -> (times, {(quantity, D): [values at times]})."""
    times, table = None, {}
    for r in _rows("drop_%s_pflbm.txt" % case):
        if r[0] == "t":
            times = [float(v) for v in r[2:]]
        else:
            table[(r[0], int(r[1]))] = [float(v) for v in r[2:]]
    return times, table
