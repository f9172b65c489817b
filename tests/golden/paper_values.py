"""Loader for paper_values.txt: the numbers the paper prints that the oracle
tests hold it to, each cited in the text file."""
import os


def load():
    path = os.path.join(os.path.dirname(__file__), "paper_values.txt")
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals
