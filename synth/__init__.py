"""Seeded synthetic inputs for the BBC large-k IVF search path.

This package produces the data every consumer shares: database vectors,
queries, request streams and the offline IVF index built over them (k-means
centroids, inverted lists, PQ codebooks and codes).  It holds none of the
search method's arithmetic: no probe scores, lookup tables, estimated
distances, bucket codebooks, collectors or re-rank.  The CPU oracle and the
CUDA library each implement the search on their own and only read what this
package generates.
"""

from .data import (  # noqa: F401
    WORKLOADS,
    Workload,
    make_workload,
    gaussian_mixture_tiny,
    sift_shaped,
    sift_iid_mixture,
    gist_shaped,
    embedding_shaped,
)
from .index import (  # noqa: F401
    IvfPqIndex,
    IvfSignIndex,
    build_ivf_pq,
    build_ivf_sign,
    kmeans,
    write_index,
)
