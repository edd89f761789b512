"""Test helper: import the library, building it in-tree when the .so is missing."""
import os


def tnlib():
    from paper_2110_14502_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    import paper_2110_14502_gb300 as T
    return T
