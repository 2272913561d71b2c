"""ORACLE -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle.so``, the plain
single-threaded FP64 C restatement of the paper's Monte Carlo scatter forward
projection (``mc_oracle.c``), and ``post.py``, the plain numpy restatement of
the smoothing and interpolation step.  It shares no code with the CUDA
library; the two meet only in the seeded inputs from ``mc_inputs``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ST_NAMES = [
    "histories", "flight_steps", "nee_steps", "nee_rays", "photo", "compton", "rayleigh", "escape",
    "max_energy_error", "limit", "sampler_fail", "e_source", "e_deposit", "e_escape", "rr_killed",
]


def build(force=False):
    """Compile the oracle with gcc (FP contraction off so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        d, i, u32, u64 = C.c_double, C.c_int, C.c_uint32, C.c_uint64
        dp = C.POINTER(C.c_double)
        L.orc_create.argtypes = [C.POINTER(P)]
        L.orc_destroy.argtypes = [P]
        L.orc_destroy.restype = None
        L.orc_load_tables.argtypes = [P, C.c_char_p]
        L.orc_load_volume.argtypes = [P, P, P, i, i, i, d, d, d]
        L.orc_set_spectrum.argtypes = [P, P, P, i]
        L.orc_set_geometry.argtypes = [P, d, d, i, i, d, d]
        L.orc_set_detector_response.argtypes = [P, P, i]
        L.orc_set_nee_mode.argtypes = [P, i]
        L.orc_set_doppler.argtypes = [P, i]
        L.orc_set_tiles.argtypes = [P, i, i]
        L.orc_set_forced.argtypes = [P, i]
        L.orc_load_mesh.argtypes = [P, P, i, P, P, i, P, P, P, i]
        L.orc_mesh_primary.argtypes = [P, d, P]
        L.orc_sample_doppler.argtypes = [P, i, d, d, u64, u64, P]
        L.orc_set_options.argtypes = [P, i, d, i, d]
        L.orc_primary.argtypes = [P, d, d, P, P]
        L.orc_scatter.argtypes = [P, d, u32, u64, u64, u64, d, u64, P, P, P, P, P]
        L.orc_march.argtypes = [P, dp, dp, d, d, d, d, dp, P, dp, C.POINTER(C.c_long)]
        L.orc_nee_pdf.argtypes = [P, i, i, d, d, dp]
        L.orc_nee_pdf.restype = d
        L.orc_kn_norm.argtypes = [d, d]
        L.orc_kn_norm.restype = d
        L.orc_sample_compton.argtypes = [d, d, u64, u64, P, P]
        L.orc_sample_rayleigh.argtypes = [P, i, d, u64, u64, P]
        L.orc_sample_incoherent.argtypes = [P, i, d, u64, u64, P]
        L.orc_philox.argtypes = [P, P, P]
        L.orc_philox.restype = None
        L.orc_stream.argtypes = [u64, u32, u64, i, P]
        L.orc_stratify.argtypes = [i, P, u64, P]
        L.orc_table.argtypes = [P, i, i, d]
        L.orc_table.restype = d
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _chk(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


class Oracle:
    """One oracle context: tables, volume, spectrum, geometry, options."""

    def __init__(self, table_path):
        self.L = lib()
        self.h = C.c_void_p()
        _chk(self.L.orc_create(C.byref(self.h)), "create")
        _chk(self.L.orc_load_tables(self.h, table_path.encode()), "load_tables")
        self.nu = self.nv = 0

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_volume(self, vol):
        mat = np.ascontiguousarray(vol["mat"], dtype=np.uint8)
        rho = np.ascontiguousarray(vol["rho"], dtype=np.uint16)
        nz, ny, nx = mat.shape
        dx, dy, dz = vol["spacing"]
        _chk(self.L.orc_load_volume(self.h, _ptr(mat), _ptr(rho), nx, ny, nz, dx, dy, dz), "load_volume")

    def set_spectrum(self, energies, weights):
        E = np.ascontiguousarray(energies, dtype=np.float32)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        _chk(self.L.orc_set_spectrum(self.h, _ptr(w), _ptr(E), len(E)), "set_spectrum")

    def load_mesh(self, mesh):
        """Triangle-mesh geometry (mc_inputs.meshes dict); replaces the volume for mesh_primary."""
        v = np.ascontiguousarray(mesh["vertices"], dtype=np.float32)
        t = np.ascontiguousarray(mesh["triangles"], dtype=np.int32)
        tb = np.ascontiguousarray(mesh["tri_body"], dtype=np.int32)
        bm = np.ascontiguousarray(mesh["body_material"], dtype=np.int32)
        br = np.ascontiguousarray(mesh["body_density"], dtype=np.float32)
        bp = np.ascontiguousarray(mesh["body_parent"], dtype=np.int32)
        _chk(self.L.orc_load_mesh(self.h, _ptr(v), len(v), _ptr(t), _ptr(tb), len(t), _ptr(bm), _ptr(br), _ptr(bp),
                                  len(bm)), "load_mesh")

    def mesh_primary(self, angle):
        Ip = np.zeros((self.nv, self.nu))
        _chk(self.L.orc_mesh_primary(self.h, float(np.float32(angle)), _ptr(Ip)), "mesh_primary")
        return Ip

    def set_doppler(self, on):
        """Doppler broadening of incoherent scatter (needs the bound tables)."""
        _chk(self.L.orc_set_doppler(self.h, int(on)), "set_doppler")

    def sample_doppler(self, mat, E, cos_t, n, seed):
        """E'/E of n Doppler-broadened incoherent scatters through cos_t."""
        out = np.zeros(n)
        _chk(self.L.orc_sample_doppler(self.h, mat, E, cos_t, n, seed, _ptr(out)), "sample_doppler")
        return out

    def set_tiles(self, tile_u, tile_v):
        """Tile-stratified point-detector pixels (tile_u x tile_v pixels per tile; 0, 0 = off)."""
        _chk(self.L.orc_set_tiles(self.h, int(tile_u), int(tile_v)), "set_tiles")

    def set_forced(self, on):
        """Forced detection: every interaction scores every pixel (of the history's tile) once."""
        _chk(self.L.orc_set_forced(self.h, int(on)), "set_forced")

    def set_nee_mode(self, mode):
        """0: score the sampled scatter type (the paper's); 1: expected value over both types."""
        _chk(self.L.orc_set_nee_mode(self.h, int(mode)), "set_nee_mode")

    def set_detector_response(self, eta):
        """eta at the table's energy nodes (keV per photon), or None for eta(E) = E."""
        if eta is None:
            _chk(self.L.orc_set_detector_response(self.h, None, 0), "set_detector_response")
            return
        e = np.ascontiguousarray(eta, dtype=np.float64)
        _chk(self.L.orc_set_detector_response(self.h, _ptr(e), len(e)), "set_detector_response")

    def set_geometry(self, sod, sdd, nu, nv, pu, pv):
        self.nu, self.nv = nu, nv
        _chk(self.L.orc_set_geometry(self.h, sod, sdd, nu, nv, pu, pv), "set_geometry")

    def set_options(self, n_split=10, rr_threshold=0.0, max_order=64, eps_face=0.0):
        _chk(self.L.orc_set_options(self.h, n_split, rr_threshold, max_order, eps_face), "set_options")

    def setup(self, wl):
        self.load_volume(wl["volume"])
        self.set_spectrum(wl["energies"], wl["weights"])
        self.set_geometry(**wl["geometry"])
        if wl.get("detector_response") is not None:
            self.set_detector_response(wl["detector_response"])

    def primary(self, angle, step):
        Ip = np.zeros((self.nv, self.nu))
        bound = np.zeros((self.nv, self.nu))
        _chk(self.L.orc_primary(self.h, float(np.float32(angle)), step, _ptr(Ip), _ptr(bound)), "primary")
        return Ip, bound

    def scatter(self, angle, n_photons, step, seed, h_begin=0, h_end=None, angle_index=0, orders=False,
                analog=False):
        h_end = n_photons if h_end is None else h_end
        P = self.nu * self.nv
        Is = np.zeros(P)
        Io = np.zeros(3 * P) if orders else None
        An = np.zeros(P) if analog else None
        A0 = np.zeros(P) if analog else None
        st = np.zeros(len(ST_NAMES))
        _chk(
            self.L.orc_scatter(self.h, float(np.float32(angle)), angle_index, n_photons, h_begin, h_end, step, seed,
                               _ptr(Is), _ptr(Io), _ptr(An), _ptr(A0), _ptr(st)),
            "scatter",
        )
        shp = (self.nv, self.nu)
        out = dict(Is=Is.reshape(shp), stats=dict(zip(ST_NAMES, st)))
        if orders:
            out["orders"] = Io.reshape(3, *shp)
        if analog:
            out["analog"] = An.reshape(shp)
            out["analog0"] = A0.reshape(shp)
        return out

    def march(self, p0, w, t0, t1, step, E):
        p0 = (C.c_double * 3)(*p0)
        w = (C.c_double * 3)(*w)
        tau = C.c_double()
        bound = C.c_double()
        rhoL = (C.c_double * 16)()
        ns = C.c_long()
        _chk(self.L.orc_march(self.h, p0, w, t0, t1, step, E, C.byref(tau), rhoL, C.byref(bound), C.byref(ns)),
             "march")
        return tau.value, np.array(rhoL[:]), bound.value, ns.value

    def nee_pdf(self, type_, mat, E, lam):
        Eo = C.c_double()
        p = self.L.orc_nee_pdf(self.h, type_, mat, E, lam, C.byref(Eo))
        return p, Eo.value

    def sample_rayleigh(self, mat, E, n, seed):
        out = np.zeros(n)
        _chk(self.L.orc_sample_rayleigh(self.h, mat, E, n, seed, _ptr(out)), "sample_rayleigh")
        return out

    def sample_incoherent(self, mat, E, n, seed):
        """cos(theta) of n incoherent scatters (with the scattering function when the tables have it)."""
        out = np.zeros(n)
        _chk(self.L.orc_sample_incoherent(self.h, mat, E, n, seed, _ptr(out)), "sample_incoherent")
        return out

    def table(self, which, mat, E):
        return self.L.orc_table(self.h, which, mat, E)


def sample_compton(E, n, seed, mec2=510.99895):
    c = np.zeros(n)
    r = np.zeros(n)
    _chk(lib().orc_sample_compton(E, mec2, n, seed, _ptr(c), _ptr(r)), "sample_compton")
    return c, r


def kn_norm(E, mec2=510.99895):
    return lib().orc_kn_norm(E, mec2)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(o))
    return o


def stream(h, angle_index, seed, n):
    o = np.zeros(n, dtype=np.uint32)
    lib().orc_stream(h, angle_index, seed, n, _ptr(o))
    return o


def stratify(S, N):
    S = np.ascontiguousarray(S, dtype=np.float64)
    M = np.zeros(len(S), dtype=np.uint64)
    _chk(lib().orc_stratify(len(S), _ptr(S), N, _ptr(M)), "stratify")
    return M
