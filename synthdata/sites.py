"""Detector sites of the HLVK network as ECEF vectors.

The paper (Sec. V) uses the four-detector network H1, L1, V1, K1 but does not list the site
coordinates. The values below are the approximate published geodetic positions (WGS-84,
zero height) and arm bearings (degrees clockwise from local North, arms taken horizontal).
They only affect how realistic the network is: every test compares two implementations that
receive the same vectors.
"""

import math

import numpy as np

# name: (latitude deg, longitude deg, x-arm bearing deg, y-arm bearing deg)
SITES = {
    "H1": (46.455147, -119.407656, 324.0000, 234.0000),
    "L1": (30.562894, -90.774242, 252.2835, 162.2835),
    "V1": (43.631414, 10.504497, 19.4326, 289.4326),
    "K1": (36.411900, 137.305600, 60.3964, 150.3964),
}

_WGS84_A = 6378137.0
_WGS84_F = 1.0 / 298.257223563


def _geodetic_to_ecef(lat_deg, lon_deg):
    lat = math.radians(lat_deg)
    lon = math.radians(lon_deg)
    e2 = _WGS84_F * (2.0 - _WGS84_F)
    n = _WGS84_A / math.sqrt(1.0 - e2 * math.sin(lat) ** 2)
    return np.array([
        n * math.cos(lat) * math.cos(lon),
        n * math.cos(lat) * math.sin(lon),
        n * (1.0 - e2) * math.sin(lat),
    ])


def _arm(lat_deg, lon_deg, bearing_deg):
    lat = math.radians(lat_deg)
    lon = math.radians(lon_deg)
    b = math.radians(bearing_deg)
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.array([-math.sin(lat) * math.cos(lon), -math.sin(lat) * math.sin(lon), math.cos(lat)])
    v = math.cos(b) * north + math.sin(b) * east
    return v / np.linalg.norm(v)


def detector_geometry(names=("H1", "L1", "V1", "K1")):
    """Return an array (D, 9): ECEF position r [m], unit x-arm, unit y-arm for each named site."""
    rows = []
    for name in names:
        lat, lon, bx, by = SITES[name]
        rows.append(np.concatenate([_geodetic_to_ecef(lat, lon), _arm(lat, lon, bx), _arm(lat, lon, by)]))
    return np.array(rows, dtype=np.float64)
