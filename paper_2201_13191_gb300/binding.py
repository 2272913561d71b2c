"""ctypes binding of include/mc.h: same entry points, argument marshalling only.

Device buffers are torch tensors on the context's CUDA device; streams are
torch streams (their raw cudaStream_t handles are passed through).  Host
arrays (angles, spectrum) are numpy arrays.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import OUT as _LIB_PATH

MC_OK = 0
_ERRORS = {
    -1: "MC_ERR_INVALID_ARG",
    -2: "MC_ERR_STATE",
    -3: "MC_ERR_CUDA",
    -4: "MC_ERR_OOM",
    -5: "MC_ERR_TIMEOUT",
    -6: "MC_ERR_LIMIT",
    -7: "MC_ERR_INTERNAL",
    -8: "MC_ERR_IO",
}
STAT_NAMES = [
    "histories", "flight_steps", "nee_steps", "nee_rays", "photo", "compton", "rayleigh", "escape", "limit",
    "sampler_fail", "transport_ms", "primary_ms",
]
EXPORTED = [
    "mc_default_options", "mc_create", "mc_destroy", "mc_set_options", "mc_last_error", "mc_load_tables",
    "mc_load_volume", "mc_set_spectrum", "mc_set_geometry", "mc_project", "mc_project_histories",
    "mc_last_stats", "mc_smooth_upsample", "mc_project_scatter_static", "mc_autotune", "mc_denoise_init",
    "mc_denoise_train_step", "mc_denoise_infer", "mc_denoise_get_layer", "mc_denoise_set_layer", "mc_denoise_save",
    "mc_denoise_load", "mc_nn_conv3x3", "mc_nn_conv3x3_wgrad", "mc_correct_iter", "mc_fdk", "mc_bin_volume",
    "mc_set_detector_response", "mc_load_mesh", "mc_line_integrals", "mc_segment", "mc_correct_images",
]


class MCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Tuning(C.Structure):
    _fields_ = [
        ("step_mm", C.c_float),
        ("block_size", C.c_int),
        ("blocks_per_sm", C.c_int),
        ("tally_mode", C.c_int),
        ("histories_per_s", C.c_double),
        ("step_error", C.c_double),
        ("rr_threshold", C.c_float),
        ("rr_fom_gain", C.c_double),
        ("tile_u", C.c_int),
        ("tile_v", C.c_int),
        ("tile_fom_gain", C.c_double),
    ]


class CorrectParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
        ("sim_nu", C.c_int), ("sim_nv", C.c_int),
        ("sim_angle_stride", C.c_int),
        ("photons", C.c_uint64),
        ("step_mm", C.c_float),
        ("seed", C.c_uint64),
        ("classes", C.c_int),
        ("class_material", C.c_int * 3),
        ("class_density0", C.c_float),
        ("e_eff_keV", C.c_float),
        ("mu_lo", C.c_float), ("mu_hi", C.c_float),
        ("primary_full_res", C.c_int),
        ("mc_bin", C.c_int),
    ]


class Options(C.Structure):
    _fields_ = [
        ("n_split", C.c_int),
        ("rr_threshold", C.c_float),
        ("max_scatter_order", C.c_int),
        ("n_batches", C.c_int),
        ("block_size", C.c_int),
        ("blocks_per_sm", C.c_int),
        ("tally_mode", C.c_int),
        ("sg_window", C.c_int),
        ("sg_order", C.c_int),
        ("cubic_a", C.c_float),
        ("denoise_mode", C.c_int),
        ("voxel_layout", C.c_int),
        ("use_graph", C.c_int),
        ("nee_mode", C.c_int),
        ("doppler", C.c_int),
        ("tile_u", C.c_int),
        ("tile_v", C.c_int),
        ("forced_detection", C.c_int),
    ]


_lib = None


def library_path():
    return _LIB_PATH


def library():
    """Load libmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise OSError(f"{_LIB_PATH} is missing: build it with paper_2201_13191_gb300.build()")
        L = C.CDLL(_LIB_PATH)
        P, i, f, u64, vp = C.c_void_p, C.c_int, C.c_float, C.c_uint64, C.c_void_p
        L.mc_default_options.argtypes = [C.POINTER(Options)]
        L.mc_default_options.restype = None
        L.mc_create.argtypes = [C.POINTER(P), i, C.POINTER(Options)]
        L.mc_destroy.argtypes = [P]
        L.mc_destroy.restype = None
        L.mc_set_options.argtypes = [P, C.POINTER(Options)]
        L.mc_last_error.argtypes = [P]
        L.mc_last_error.restype = C.c_char_p
        L.mc_load_tables.argtypes = [P, C.c_char_p]
        L.mc_load_volume.argtypes = [P, vp, vp, i, i, i, f, f, f, i, vp]
        L.mc_set_spectrum.argtypes = [P, vp, vp, i]
        L.mc_set_geometry.argtypes = [P, f, f, i, i, f, f]
        L.mc_project.argtypes = [P, vp, i, u64, f, u64, vp, vp, vp, vp]
        L.mc_project_histories.argtypes = [P, vp, i, u64, u64, u64, f, u64, vp, vp]
        L.mc_last_stats.argtypes = [P, C.POINTER(C.c_double), i]
        L.mc_smooth_upsample.argtypes = [P, vp, i, vp, i, i, vp, i, vp, i, i, vp]
        L.mc_project_scatter_static.argtypes = [P, vp, i, u64, f, u64, vp, vp]
        L.mc_autotune.argtypes = [P, vp, i, u64, f, f, f, C.POINTER(Tuning), vp]
        fp = C.POINTER(C.c_float)
        ip = C.POINTER(C.c_int)
        L.mc_denoise_init.argtypes = [P, i, i, i, u64]
        L.mc_denoise_train_step.argtypes = [P, vp, vp, i, f, fp, vp]
        L.mc_denoise_infer.argtypes = [P, vp, vp, i, vp]
        L.mc_denoise_get_layer.argtypes = [P, i, vp, vp, vp, vp, ip, ip]
        L.mc_denoise_set_layer.argtypes = [P, i, vp, vp]
        L.mc_denoise_save.argtypes = [P, C.c_char_p]
        L.mc_denoise_load.argtypes = [P, C.c_char_p, i]
        L.mc_nn_conv3x3.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, i, vp, vp]
        L.mc_nn_conv3x3_wgrad.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp, vp]
        L.mc_correct_iter.argtypes = [P, vp, vp, i, vp, i, i, i, C.POINTER(CorrectParams), vp, vp, vp, vp]
        L.mc_fdk.argtypes = [P, vp, i, vp, i, i, i, i, i, f, f, f, vp, vp]
        L.mc_bin_volume.argtypes = [P, vp, vp, i, i, i, f, vp, vp, vp]
        L.mc_line_integrals.argtypes = [P, vp, vp, i, i, i, vp, vp]
        L.mc_segment.argtypes = [P, vp, i, i, i, i, vp, f, f, f, f, vp, vp, vp, vp, vp]
        L.mc_correct_images.argtypes = [P, vp, vp, vp, f, C.c_size_t, vp, vp]
        L.mc_set_detector_response.argtypes = [P, vp, i]
        L.mc_load_mesh.argtypes = [P, vp, i, vp, vp, i, vp, vp, vp, i]
        _lib = L
    return _lib


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _t_ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def conv3x3(x, w, bias=None, relu=False, out_f32=True, stream=None):
    """Tensor-core 3x3 convolution (mc_nn_conv3x3): x BF16 [n][h][w][cin] (torch.bfloat16 on the device),
    w BF16 [cout][9][cin], bias FP32 [cout] or None; returns FP32 or BF16 [n][h][w][cout]."""
    import torch

    n, h, wd, cin = x.shape
    cout = w.shape[0]
    y = torch.empty((n, h, wd, cout), dtype=torch.float32 if out_f32 else torch.bfloat16, device=x.device)
    err = torch.zeros(1, dtype=torch.int32, device=x.device)
    rc = library().mc_nn_conv3x3(_t_ptr(x.contiguous()), _t_ptr(w.contiguous()), _t_ptr(bias), _t_ptr(y), n, h, wd,
                                 cin, cout, int(relu), int(out_f32), _t_ptr(err), _stream_handle(stream))
    if rc != MC_OK:
        raise MCError(rc, "mc_nn_conv3x3 failed")
    torch.cuda.synchronize()
    if int(err.item()):
        raise MCError(-5, "a tensor-core wait gave up")
    return y


def conv3x3_wgrad(x, dy, splits=8, stream=None):
    """Weight gradient on the tensor cores (mc_nn_conv3x3_wgrad): FP32 [cout][9][cin]."""
    import torch

    n, h, wd, cin = x.shape
    cout = dy.shape[-1]
    dw = torch.zeros((cout, 9, cin), dtype=torch.float32, device=x.device)
    err = torch.zeros(1, dtype=torch.int32, device=x.device)
    rc = library().mc_nn_conv3x3_wgrad(_t_ptr(x.contiguous()), _t_ptr(dy.contiguous()), _t_ptr(dw), n, h, wd, cin,
                                       cout, splits, _t_ptr(err), _stream_handle(stream))
    if rc != MC_OK:
        raise MCError(rc, "mc_nn_conv3x3_wgrad failed")
    torch.cuda.synchronize()
    if int(err.item()):
        raise MCError(-5, "a tensor-core wait gave up")
    return dw


def _stream_handle(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """One mc_ctx on a CUDA device.  Method names follow the C entry points."""

    def __init__(self, device=0, **options):
        import torch

        self.torch = torch
        self.L = library()
        self.device = torch.device("cuda", device)
        opt = Options()
        self.L.mc_default_options(C.byref(opt))
        for k, v in options.items():
            setattr(opt, k, v)
        self.opt = opt
        self.h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.L.mc_create(C.byref(self.h), device, C.byref(opt))
        if rc != MC_OK:
            raise MCError(rc, "mc_create failed")
        self.nu = self.nv = 0

    def _check(self, rc, allow_limit=False):
        if rc == MC_OK or (allow_limit and rc == -6):
            return rc
        raise MCError(rc, self.L.mc_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.L.mc_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **options):
        for k, v in options.items():
            setattr(self.opt, k, v)
        self._check(self.L.mc_set_options(self.h, C.byref(self.opt)))

    def load_tables(self, path):
        self._check(self.L.mc_load_tables(self.h, str(path).encode()))

    def load_volume(self, mat, rho_fp16, spacing, stream=None):
        """mat: uint8 [nz][ny][nx]; rho_fp16: uint16 (binary16 bits) or float16, numpy (host) or torch (host/device)."""
        torch = self.torch
        if isinstance(mat, np.ndarray):
            mat = np.ascontiguousarray(mat, dtype=np.uint8)
            rho = np.ascontiguousarray(rho_fp16).view(np.uint16)
            nz, ny, nx = mat.shape
            pm, pr, dev = _np_ptr(mat), _np_ptr(rho), 0
        else:
            mat = mat.contiguous()
            rho = rho_fp16.contiguous()
            nz, ny, nx = mat.shape
            pm, pr, dev = _t_ptr(mat), _t_ptr(rho), int(mat.is_cuda)
        dx, dy, dz = spacing
        self._check(
            self.L.mc_load_volume(self.h, pm, pr, nx, ny, nz, dx, dy, dz, dev, _stream_handle(stream))
        )
        self._keep = (mat, rho)

    def set_spectrum(self, energies, weights):
        E = np.ascontiguousarray(energies, dtype=np.float32)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        self._check(self.L.mc_set_spectrum(self.h, _np_ptr(w), _np_ptr(E), len(E)))

    def set_geometry(self, sod, sdd, nu, nv, pu, pv):
        self.nu, self.nv = nu, nv
        self._check(self.L.mc_set_geometry(self.h, sod, sdd, nu, nv, pu, pv))

    def load_mesh(self, mesh):
        """Triangle-mesh geometry (an mc_inputs.meshes dict of host arrays); primary images only."""
        v = np.ascontiguousarray(mesh["vertices"], dtype=np.float32)
        t = np.ascontiguousarray(mesh["triangles"], dtype=np.int32)
        tb = np.ascontiguousarray(mesh["tri_body"], dtype=np.int32)
        bm = np.ascontiguousarray(mesh["body_material"], dtype=np.int32)
        br = np.ascontiguousarray(mesh["body_density"], dtype=np.float32)
        bp = np.ascontiguousarray(mesh["body_parent"], dtype=np.int32)
        self._check(self.L.mc_load_mesh(self.h, _np_ptr(v), len(v), _np_ptr(t), _np_ptr(tb), len(t), _np_ptr(bm),
                                        _np_ptr(br), _np_ptr(bp), len(bm)))

    def set_detector_response(self, eta):
        """eta at the table's energy nodes (keV per photon, host), or None for eta(E) = E."""
        if eta is None:
            self._check(self.L.mc_set_detector_response(self.h, None, 0))
            return
        e = np.ascontiguousarray(eta, dtype=np.float64)
        self._check(self.L.mc_set_detector_response(self.h, _np_ptr(e), len(e)))

    def setup(self, wl):
        v = wl["volume"]
        self.load_volume(v["mat"], v["rho"], v["spacing"])
        self.set_spectrum(wl["energies"], wl["weights"])
        self.set_geometry(**wl["geometry"])
        if wl.get("detector_response") is not None:
            self.set_detector_response(wl["detector_response"])

    def empty_images(self, n_angles):
        return self.torch.empty((n_angles, self.nv, self.nu), dtype=self.torch.float32, device=self.device)

    def project(self, angles, n_photons, step_mm, seed, primary=True, scatter=True, variance=False, out=None,
                stream=None, allow_limit=False):
        """Returns dict(primary=, scatter=, variance=) of [n_angles][nv][nu] FP32 device tensors."""
        a = np.ascontiguousarray(np.atleast_1d(angles), dtype=np.float32)
        out = dict(out or {})
        if primary and out.get("primary") is None:
            out["primary"] = self.empty_images(len(a))
        if scatter and out.get("scatter") is None:
            out["scatter"] = self.empty_images(len(a))
        if variance and out.get("variance") is None:
            out["variance"] = self.empty_images(len(a))
        rc = self.L.mc_project(
            self.h, _np_ptr(a), len(a), int(n_photons), float(step_mm), int(seed),
            _t_ptr(out.get("primary") if primary else None), _t_ptr(out.get("scatter") if scatter else None),
            _t_ptr(out.get("variance") if variance else None), _stream_handle(stream),
        )
        self._check(rc, allow_limit)
        return out

    def project_histories(self, angles, n_photons, h_begin, h_count, step_mm, seed, out=None, stream=None):
        a = np.ascontiguousarray(np.atleast_1d(angles), dtype=np.float32)
        if out is None:
            out = self.empty_images(len(a))
        rc = self.L.mc_project_histories(
            self.h, _np_ptr(a), len(a), int(n_photons), int(h_begin), int(h_count), float(step_mm), int(seed),
            _t_ptr(out), _stream_handle(stream),
        )
        self._check(rc)
        return out

    def project_scatter_static(self, angles, n_photons, step_mm, seed, out=None, stream=None, allow_limit=False):
        """Scatter image through the entry point that allocates nothing (its
        scratch is a fixed array inside the library); out is allocated here by
        torch only when the caller does not pass one."""
        a = np.ascontiguousarray(np.atleast_1d(angles), dtype=np.float32)
        if out is None:
            out = self.empty_images(len(a))
        rc = self.L.mc_project_scatter_static(
            self.h, _np_ptr(a), len(a), int(n_photons), float(step_mm), int(seed), _t_ptr(out), _stream_handle(stream)
        )
        self._check(rc, allow_limit)
        return out

    def autotune(self, angles, probe_photons, step_min, step_max, step_tol, stream=None, cache=None, cache_key=None):
        """Run mc_autotune; with cache (a JSON path) and cache_key, reuse an
        earlier result for the same key instead of tuning again."""
        import json

        if cache and cache_key and os.path.exists(cache):
            with open(cache) as f:
                saved = json.load(f).get(cache_key)
            if saved:
                opt = dict(block_size=saved["block_size"], blocks_per_sm=saved["blocks_per_sm"],
                           tally_mode=saved["tally_mode"], rr_threshold=saved.get("rr_threshold", 0.0))
                if saved.get("tile_u", 0) > 0:
                    opt.update(tally_mode=4, tile_u=saved["tile_u"], tile_v=saved["tile_v"])
                self.set_options(**opt)
                return saved
        a = np.ascontiguousarray(np.atleast_1d(angles), dtype=np.float32)
        t = Tuning()
        self._check(self.L.mc_autotune(self.h, _np_ptr(a), len(a), int(probe_photons), float(step_min),
                                       float(step_max), float(step_tol), C.byref(t), _stream_handle(stream)))
        self.opt.block_size, self.opt.blocks_per_sm, self.opt.tally_mode = t.block_size, t.blocks_per_sm, t.tally_mode
        self.opt.rr_threshold = t.rr_threshold
        if t.tile_u > 0:
            self.opt.tally_mode, self.opt.tile_u, self.opt.tile_v = 4, t.tile_u, t.tile_v
        res = {k: getattr(t, k) for k, _ in Tuning._fields_}
        if cache and cache_key:
            data = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    data = json.load(f)
            data[cache_key] = res
            with open(cache, "w") as f:
                json.dump(data, f, indent=1)
        return res

    # ---- correction plumbing
    def fdk(self, p, angles, NU, NV, grid, stream=None):
        """FDK of line integrals p (device [n][NV][NU]); grid = (nx, ny, nz, dx, dy, dz) -> [nz][ny][nx]."""
        nx, ny, nz, dx, dy, dz = grid
        a = np.ascontiguousarray(angles, dtype=np.float32)
        vol = self.torch.empty((max(nz, 1), max(ny, 1), max(nx, 1)), dtype=self.torch.float32, device=self.device)
        self._check(self.L.mc_fdk(self.h, _t_ptr(p.contiguous()), len(a), _np_ptr(a), NU, NV, nx, ny, nz, dx, dy, dz,
                                  _t_ptr(vol), _stream_handle(stream)))
        return vol

    def bin_volume(self, mat, rho, e_eff_keV, stream=None):
        """2x2x2 down-sampling of a segmented volume (device uint8 mat, int16/uint16 binary16 rho, [nz][ny][nx],
        even dims) for the Monte Carlo step -> (mat, rho) device tensors [nz/2][ny/2][nx/2]."""
        torch = self.torch
        nz, ny, nx = mat.shape
        mo = torch.empty((nz // 2, ny // 2, nx // 2), dtype=torch.uint8, device=mat.device)
        ro = torch.empty((nz // 2, ny // 2, nx // 2), dtype=torch.int16, device=mat.device)
        self._check(self.L.mc_bin_volume(self.h, _t_ptr(mat.contiguous()), _t_ptr(rho.contiguous()), nx, ny, nz,
                                         float(e_eff_keV), _t_ptr(mo), _t_ptr(ro), _stream_handle(stream)))
        return mo, ro

    def line_integrals(self, I, I0, stream=None):
        """a = -ln(I / I0) (mc_line_integrals): I device [n][NV][NU], I0 device [NV][NU]."""
        I = I.contiguous()
        n, NV, NU = I.shape
        a = self.torch.empty_like(I)
        self._check(self.L.mc_line_integrals(self.h, _t_ptr(I), _t_ptr(I0.contiguous()), n, NU, NV, _t_ptr(a),
                                             _stream_handle(stream)))
        return a

    def segment(self, vol, classes, class_material, class_density0, e_eff_keV, mu_lo, mu_hi, stream=None):
        """Otsu segmentation and class -> material / density (mc_segment) of a device FP32 volume
        [nz][ny][nx]; returns (mat uint8, rho int16 binary16 bits) device tensors, the 256-bin histogram and
        the two thresholds (numpy)."""
        torch = self.torch
        vol = vol.contiguous()
        nz, ny, nx = vol.shape
        mat = torch.empty((nz, ny, nx), dtype=torch.uint8, device=vol.device)
        rho = torch.empty((nz, ny, nx), dtype=torch.int16, device=vol.device)
        cm = np.zeros(3, np.int32)
        cm[: len(class_material)] = class_material
        hist = np.zeros(256, np.uint32)
        thr = np.zeros(2, np.int32)
        self._check(self.L.mc_segment(self.h, _t_ptr(vol), nx, ny, nz, int(classes), _np_ptr(cm),
                                      float(class_density0), float(e_eff_keV), float(mu_lo), float(mu_hi),
                                      _np_ptr(hist), _np_ptr(thr), _t_ptr(mat), _t_ptr(rho), _stream_handle(stream)))
        return mat, rho, hist, thr

    def correct_images(self, a, ip, is_, is_scale=1.0, stream=None):
        """Eq. (Correction) per element (mc_correct_images): c = a - ln(Ip / (Ip + s Is))."""
        a = a.contiguous()
        c = self.torch.empty_like(a)
        self._check(self.L.mc_correct_images(self.h, _t_ptr(a), _t_ptr(ip.contiguous()), _t_ptr(is_.contiguous()),
                                             float(is_scale), a.numel(), _t_ptr(c), _stream_handle(stream)))
        return c

    def correct_iter(self, raw_I, I0, angles, NU, NV, n_iter, prm, stream=None):
        """Iterative scatter correction; returns (corrected line integrals, last volume, seconds per iteration)."""
        a = np.ascontiguousarray(angles, dtype=np.float32)
        out = self.torch.empty_like(raw_I)
        vol = self.torch.empty((prm.nz, prm.ny, prm.nx), dtype=self.torch.float32, device=self.device)
        secs = np.zeros(max(n_iter, 1))
        self._check(self.L.mc_correct_iter(self.h, _t_ptr(raw_I.contiguous()), _t_ptr(I0.contiguous()), len(a),
                                           _np_ptr(a), NU, NV, n_iter, C.byref(prm), _t_ptr(out), _t_ptr(vol),
                                           _np_ptr(secs), _stream_handle(stream)))
        return out, vol, list(secs[:n_iter])

    # ---- learned denoiser
    def denoise_init(self, height, width, max_batch, seed=0):
        self._check(self.L.mc_denoise_init(self.h, height, width, max_batch, seed))

    def denoise_train_step(self, noisy, clean, lr, stream=None):
        """noisy, clean: device FP32 [n][h][w]; returns the batch loss before the step."""
        loss = C.c_float()
        n = noisy.shape[0]
        self._check(self.L.mc_denoise_train_step(self.h, _t_ptr(noisy.contiguous()), _t_ptr(clean.contiguous()), n,
                                                 float(lr), C.byref(loss), _stream_handle(stream)))
        return loss.value

    def denoise_infer(self, images, out=None, stream=None):
        images = images.contiguous()
        if out is None:
            out = self.torch.empty_like(images)
        self._check(self.L.mc_denoise_infer(self.h, _t_ptr(images), _t_ptr(out), images.shape[0],
                                            _stream_handle(stream)))
        return out

    def denoise_layer(self, i):
        ci, co = C.c_int(), C.c_int()
        self._check(self.L.mc_denoise_get_layer(self.h, i, None, None, None, None, C.byref(ci), C.byref(co)))
        w = np.zeros((co.value, 9, ci.value), np.float32)
        b = np.zeros(co.value, np.float32)
        gw = np.zeros_like(w)
        gb = np.zeros_like(b)
        self._check(self.L.mc_denoise_get_layer(self.h, i, _np_ptr(w), _np_ptr(b), _np_ptr(gw), _np_ptr(gb),
                                                C.byref(ci), C.byref(co)))
        return w, b, gw, gb

    def denoise_set_layer(self, i, w, b):
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        self._check(self.L.mc_denoise_set_layer(self.h, i, _np_ptr(w), _np_ptr(b)))

    def denoise_save(self, path):
        self._check(self.L.mc_denoise_save(self.h, str(path).encode()))

    def denoise_load(self, path, max_batch=16):
        self._check(self.L.mc_denoise_load(self.h, str(path).encode(), max_batch))

    def last_stats(self):
        buf = (C.c_double * len(STAT_NAMES))()
        self._check(self.L.mc_last_stats(self.h, buf, len(STAT_NAMES)))
        return dict(zip(STAT_NAMES, list(buf)))

    def smooth_upsample(self, images, in_angles, out_angles, NU, NV, out=None, stream=None):
        torch = self.torch
        images = images.contiguous()
        n_in, nv, nu = images.shape
        ia = np.ascontiguousarray(np.atleast_1d(in_angles), dtype=np.float32)
        oa = np.ascontiguousarray(np.atleast_1d(out_angles), dtype=np.float32)
        if out is None:
            out = torch.empty((len(oa), NV, NU), dtype=torch.float32, device=images.device)
        self._check(
            self.L.mc_smooth_upsample(
                self.h, _t_ptr(images), n_in, _np_ptr(ia), nu, nv, _t_ptr(out), len(oa), _np_ptr(oa), NU, NV,
                _stream_handle(stream),
            )
        )
        return out
