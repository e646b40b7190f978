"""Readers for the text fixtures under tests/golden (values transcribed from
the paper; each file's header names the figure or passage it comes from)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def grid(name, inf=-1):
    """Numeric grid; 'inf' cells become `inf` (an int sentinel)."""
    rows = []
    for line in _lines(name):
        rows.append([inf if c == "inf" else int(c) for c in line.split()])
    return np.array(rows, dtype=np.int64)


def keyed(name):
    """Lines of the form 'key v1 v2 ...' as a dict of string lists."""
    out = {}
    for line in _lines(name):
        parts = line.split()
        out[parts[0]] = parts[1:]
    return out


def pairs(name):
    """Grid of 'dy,dx' cells ('-' = none) as two int arrays (-1 = none)."""
    dy, dx = [], []
    for line in _lines(name):
        cells = line.split()
        dy.append([-1 if c == "-" else int(c.split(",")[0]) for c in cells])
        dx.append([-1 if c == "-" else int(c.split(",")[1]) for c in cells])
    return np.array(dy, dtype=np.int64), np.array(dx, dtype=np.int64)


def sections(name):
    """A fixture of named sections: a line holding one word starts a section,
    the lines after it are its grid rows.  Returns {name: [row strings]}."""
    out, cur = {}, None
    for line in _lines(name):
        if len(line.split()) == 1 and not line[0].isdigit() and line not in ("-",):
            cur = line
            out[cur] = []
        else:
            out[cur].append(line)
    return out


def pair_rows(rows):
    """'dy,dx' cells of the given rows ('-' = none) as two int arrays."""
    dy = [[-1 if c == "-" else int(c.split(",")[0]) for c in r.split()] for r in rows]
    dx = [[-1 if c == "-" else int(c.split(",")[1]) for c in r.split()] for r in rows]
    return np.array(dy, dtype=np.int64), np.array(dx, dtype=np.int64)


def six_object_mask():
    """Fig. 18(a) as a uint8 mask (1 = object)."""
    g = grid("fig18a_init.txt")
    return (g == 0).astype(np.uint8)
