"""Structure of the facility-location generator that the evaluation and
sampling layouts rely on (CPU only): one-hot groups and closure lists are
arithmetic progressions (generated in the samplers, not read), the linking
rows x_ij <= y_i are two-variable rows around the hubs y_i whose members
step by the number of facilities (runs, and consecutive hubs side by side),
and every facility column has one entry per customer (long columns of one
length, in interleaved slices).  If the generator changes, these layouts
fall back to the general ones; this test says so first."""
import numpy as np

from paper_2510_27117_b300 import workloads as W


def _arith(idx):
    d = np.diff(idx)
    return d.size == 0 or (d[0] > 0 and np.all(d == d[0]))


def test_facility_structure_matches_the_fast_layouts():
    nf, nc = 40, 300
    inst = W.facility_location(nf=nf, nc=nc, idx=3)
    gp, gi = inst.groups
    assert gp.size - 1 == nc
    for g in range(nc):                      # customer j: x_j0 .. x_j(nf-1), step 1
        mem = gi[gp[g]:gp[g + 1]]
        assert mem.size == nf and _arith(mem) and mem[1] - mem[0] == 1
    rv, rp, ri = inst.closure
    assert np.array_equal(rv, np.arange(nf))
    for q in range(nf):                      # y_i's list: x_ij over j, step nf
        lst = ri[rp[q]:rp[q + 1]]
        assert lst.size == nc and _arith(lst) and lst[1] - lst[0] == nf
    A = inst.A.tocsr()
    assert A.shape[0] == nf * nc
    rows_of_hub = {}
    for r in range(A.shape[0]):
        cols = A.indices[A.indptr[r]:A.indptr[r + 1]]
        vals = A.data[A.indptr[r]:A.indptr[r + 1]]
        assert cols.size == 2
        hub = int(cols[np.argmax(vals)])     # y_i - x_ij >= 0: +1 on the hub
        assert hub < nf
        rows_of_hub.setdefault(hub, []).append(int(cols[np.argmin(vals)]))
    for i, members in rows_of_hub.items():
        m = np.sort(np.array(members))
        assert m.size == nc and _arith(m) and m[1] - m[0] == nf
        assert m[0] - i == nf                 # v1 - v2 equal over the hubs
    colcount = np.bincount(A.indices, minlength=inst.n)[:nf]
    assert np.all(colcount == nc)            # long columns of one length
