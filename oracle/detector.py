"""Detector response of the network (Sec. 4.1.1 three-detector analysis).

A detector with unit arm vectors x, y has the response tensor
D = (x x^T - y y^T) / 2.  A source at right ascension alpha and declination delta
(Earth-fixed longitude phi = alpha - gmst, polar angle theta = pi/2 - delta) with
polarisation angle psi defines the wave-frame axes
  X = ( sin phi cos psi - sin psi cos phi cos theta,
       -cos phi cos psi - sin psi sin phi cos theta,
        sin psi sin theta )
  Y = (-sin phi sin psi - cos psi cos phi cos theta,
        cos phi sin psi - cos psi sin phi cos theta,
        sin theta cos psi )
and the polarisation tensors e+ = X X^T - Y Y^T, ex = X Y^T + Y X^T, so that
F+ = D : e+ and Fx = D : ex.  The signal reaches a vertex r a time
dt = -(r . n) / c after the geocentre, n the unit vector toward the source.
"""
import math

import numpy as np

from .constants import C_SI


def source_direction(ra: float, dec: float, gmst: float) -> np.ndarray:
    phi = ra - gmst
    return np.array([math.cos(dec) * math.cos(phi), math.cos(dec) * math.sin(phi), math.sin(dec)])


def wave_axes(ra: float, dec: float, psi: float, gmst: float):
    phi = ra - gmst
    theta = 0.5 * math.pi - dec
    sp, cp = math.sin(phi), math.cos(phi)
    st, ct = math.sin(theta), math.cos(theta)
    ss, cs = math.sin(psi), math.cos(psi)
    X = np.array([sp * cs - ss * cp * ct, -(cp * cs + ss * sp * ct), ss * st])
    Y = np.array([-sp * ss - cs * cp * ct, cp * ss - cs * sp * ct, st * cs])
    return X, Y


def antenna_pattern(x_arm, y_arm, ra, dec, psi, gmst):
    """(F+, Fx) of one detector."""
    x_arm = np.asarray(x_arm, dtype=np.float64)
    y_arm = np.asarray(y_arm, dtype=np.float64)
    D = 0.5 * (np.outer(x_arm, x_arm) - np.outer(y_arm, y_arm))
    X, Y = wave_axes(ra, dec, psi, gmst)
    e_plus = np.outer(X, X) - np.outer(Y, Y)
    e_cross = np.outer(X, Y) + np.outer(Y, X)
    return float(np.sum(D * e_plus)), float(np.sum(D * e_cross))


def time_delay(vertex, ra, dec, gmst) -> float:
    """Arrival time at the vertex minus arrival time at the geocentre [s]."""
    n = source_direction(ra, dec, gmst)
    return -float(np.dot(np.asarray(vertex, dtype=np.float64), n)) / C_SI
