"""Writes box_modes.json: the lowest acoustic modes of two rigid-walled boxes (the 1.0 x 0.8 x 0.6 m
test box and the 2.5 x 1.4 x 1.2 m cabin), c = 340 m/s, as closed forms -- no solver involved:

* continuum (Neumann walls): f_lmn = c/2 sqrt((l/Lx)^2 + (m/Ly)^2 + (n/Lz)^2);
* discrete Q1 lattice with N_a cells per axis: the tensor-cosine eigenvalues of K v = lam M v,
  lam = sum_a (6/h_a^2)(1 - cos t_a)/(2 + cos t_a), t_a = pi l_a / N_a, f = c sqrt(lam) / (2 pi).

Run from the repository root: python tests/golden/make_box_modes.py
"""
import itertools
import json
import math
import os

C = 340.0
BOXES = {"box": ((1.0, 0.8, 0.6), (20, 16, 12)), "cabin": ((2.5, 1.4, 1.2), (24, 14, 12))}


def lam1(l, n, h):
    t = math.pi * l / n
    return (6.0 / h ** 2) * (1.0 - math.cos(t)) / (2.0 + math.cos(t))


def modes(L, N, count=8):
    out = []
    for lmn in itertools.product(range(4), repeat=3):
        if lmn == (0, 0, 0):
            continue
        fc = C / 2.0 * math.sqrt(sum((q / La) ** 2 for q, La in zip(lmn, L)))
        lam = sum(lam1(q, Na, La / Na) for q, Na, La in zip(lmn, N, L))
        out.append({"lmn": list(lmn), "f_continuum": fc, "f_discrete": C * math.sqrt(lam) / (2 * math.pi)})
    out.sort(key=lambda d: d["f_discrete"])
    return out[:count]


def main():
    data = {"c": C, "boxes": {k: {"L": list(L), "cells": list(N), "modes": modes(L, N)} for k, (L, N) in BOXES.items()}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "box_modes.json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    return data


if __name__ == "__main__":
    main()
