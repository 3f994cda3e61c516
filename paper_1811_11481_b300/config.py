"""Default configuration of the track finder and the refit.

The paper gives the structure of the method but no cut values; every number
here is a reading (window sizes, pick-up and outlier cuts, miss limits,
seed covariances), chosen for cluster errors of 0.1 cm and 152 pad rows.
"""
import math

import numpy as np

DEFAULT_PARAMS = dict(
    sigma=0.1,               # cluster position error (cm), y and z
    shared_scale=2.0,        # error scale of clusters flagged as shared (Sec. 3)
    nb_wy=0.5,               # neighbour window offset in y (cm)
    nb_wz=0.5,               # neighbour window offset in z (cm)
    nb_teta=float(np.float32(math.sinh(1.0))),  # eta window |eta| <= 1 (Sec. 4)
    nb_ty=1.0,               # direction window |tan(phi)| <= 1 in y
    nb_dmax=0.5,             # max squared deviation from the straight line (cm^2)
    chi2_pick=16.0,          # pick-up cut on the normalised distance
    max_miss=4,              # consecutive empty rows that end following
    max_gap=4,               # largest row gap inside an emitted track
    min_track_hits=10,       # minimum clusters of a track
    s_max=0.95,              # |sin(phi)| limit of the propagation
    inward_cov_scale=4.0,    # covariance inflation before the inward pass
    c0t=(0.01, 0.01, 1.0, 1.0, 100.0),   # seed covariance of the tracklet fit
    c0r=(1.0, 1.0, 0.1, 0.1, 10.0),      # covariance at the start of each refit pass
    chi2_out=25.0,           # outlier cut on the predicted chi2 (Sec. 3)
    min_acc_reject=5,        # accepted clusters before rejection starts
    refit_inflate=100.0,     # covariance inflation between refit passes
    seed_max_hits=10,        # chain hits in the seed fit (Sec. 2: segments of 4-10 hits)
    chi2_merge=30.0,         # segment-merging cut on the 5-parameter chi2 (Sec. 2, phase 2)
    split_scale=1.5,         # error scales of the other special clusters in the refit (Sec. 3)
    single_row_scale=1.5,
    single_time_scale=1.5,
    edge_scale=2.0,
)

# flag bits of a cluster (Sec. 3 lists the special cluster types)
FLAG_SPLIT = 0x01
FLAG_SINGLE_ROW = 0x02
FLAG_SINGLE_TIME = 0x04
FLAG_EDGE = 0x08
FLAG_SHARED = 0x10


def default_params():
    return dict(DEFAULT_PARAMS)
