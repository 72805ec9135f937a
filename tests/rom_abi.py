"""Flatten an oracle ``RomSet`` into the arrays of the libsfm C ABI
(``include/sfm.h``), and push it into a handle."""
import numpy as np


def abi_arrays(rs):
    topo = rs.topo
    coeffs = np.concatenate([np.concatenate([rs.Gamma[s].ravel(), rs.Gammahat[s].ravel()])
                             for s in range(rs.nsub)])
    sp_shot, sp_sub, srows = [], [], []
    for q in range(rs.nshots):
        for s in sorted(rs.src[q]):
            sp_shot.append(q)
            sp_sub.append(s)
            srows.append(rs.src[q][s].ravel())
    rp_rec, rp_sub, rrows = [], [], []
    for r in range(rs.nrec):
        for s in sorted(rs.rec[r]):
            rp_rec.append(r)
            rp_sub.append(s)
            rrows.append(rs.rec[r][s].ravel())
    cat = lambda x: np.concatenate(x) if x else np.zeros(0)
    return dict(k_sub=np.asarray(rs.k), m_face=topo.mf, nbr=topo.nbr, coeffs=coeffs,
                src=(rs.nshots, sp_shot, sp_sub, cat(srows)),
                rec=(rs.nrec, rp_rec, rp_sub, cat(rrows)))


def load_into(sfm, h, rs):
    a = abi_arrays(rs)
    sfm.sfm_set_topology(h, a["k_sub"], a["m_face"], a["nbr"])
    sfm.sfm_set_coeffs(h, a["coeffs"])
    sfm.sfm_set_sources(h, *a["src"])
    sfm.sfm_set_receivers(h, *a["rec"])
    return a
