"""The source order of bc_compute with bc_options.source_order = 2, recomputed
from oracle BFS levels: sources stably sorted by their distances to the 32
first relabelled vertices (the 32 highest-degree ones), the first landmark's
distance most significant, unreached = 0xFFFF."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

LANDMARKS = 32


def grouped_order(g, perm, src, threads: int = 1) -> np.ndarray:
    """Indices into src in grouped order; perm = relabelled -> original ids (bc_graph_export)."""
    src = np.asarray(src)

    def levels(h):
        return oracle.source_detail(g.off, g.adj, int(h))["level"][: g.n][src]

    with ThreadPoolExecutor(max(1, threads)) as ex:
        lv = np.stack(list(ex.map(levels, perm[:LANDMARKS])))  # [32][nsrc]
    keys = np.where(lv < 0, 0xFFFF, lv)
    return np.lexsort(tuple(keys[j] for j in range(LANDMARKS - 1, -1, -1)))
