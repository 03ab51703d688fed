"""Python binding of include/gbnn.h (argument marshalling only) and the
warm-start network built from it.

The network is a 4-level convolutional encoder-decoder (32-64-128-256
channels, 3x3 kernels, ReLU, 2x2 average pooling, nearest upsampling, skip
concatenations) with bfloat16 weights and activations and FP32 accumulation.
Every layer, every gradient and the Adam update run in the library's
tensor-core kernels; torch tensors only hold device memory.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbm

_sig_done = False


def _lib():
    global _sig_done
    lib = lbm.load_library()
    if not _sig_done:
        vp, i, f, ll, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong, ctypes.c_size_t
        sig = {
            "gbnn_conv3x3_fwd": [vp, i, vp, vp, vp, i, vp, i, i, i, i, i, i, i, vp],
            "gbnn_flip_weights": [vp, vp, i, i, vp],
            "gbnn_conv3x3_dgrad": [vp, i, vp, vp, i, vp, i, i, i, i, i, i, vp],
            "gbnn_conv3x3_wgrad": [vp, i, vp, i, vp, vp, i, i, i, i, i, i, vp],
            "gbnn_avgpool2": [vp, i, vp, i, i, i, i, i, vp],
            "gbnn_avgpool2_bwd": [vp, i, vp, i, vp, i, i, i, i, i, i, vp],
            "gbnn_upsample2": [vp, i, vp, i, i, i, i, i, vp],
            "gbnn_upsample2_bwd": [vp, i, vp, i, i, i, i, i, vp],
            "gbnn_mse": [vp, i, vp, vp, vp, i, ll, i, f, vp, vp],
            "gbnn_adam": [vp, vp, vp, vp, vp, ll, f, f, f, f, i, vp],
            "gbnn_encode_input": [vp, f, f, f, f, i, i, vp, vp],
            "gbnn_encode_target": [vp, vp, vp, vp, ll, f, f, f, vp, vp, vp],
            "gbnn_decode_output": [vp, i, vp, ll, f, f, f, vp, vp, vp, vp],
            "gbnn_fill_zero": [vp, sz, vp],
            "gbnn_set_conv_impl": [i],
            "gbnn_status": [i],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        lib.gbnn_conv_impl.restype = ctypes.c_int
        lib.gbnn_conv_impl.argtypes = []
        _sig_done = True
    return lib


def _ck(rc, where):
    if rc != 0:
        raise RuntimeError(f"{where} failed ({rc})")


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s(stream):
    """The CUDA stream of a torch stream; None means torch's current stream,
    so kernels stay ordered with the torch operations around them."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


IMPL_AUTO, IMPL_MMA_SYNC, IMPL_TCGEN05 = 0, 1, 2


def set_conv_impl(impl: int):
    """Convolution kernels for later calls: IMPL_AUTO (tcgen05 where the
    shape is taken, else mma.sync), IMPL_MMA_SYNC or IMPL_TCGEN05 (required)."""
    _ck(_lib().gbnn_set_conv_impl(int(impl)), "gbnn_set_conv_impl")


def conv_impl() -> int:
    return int(_lib().gbnn_conv_impl())


def status(reset: bool = False) -> int:
    """Device status of the tensor-core kernels: 1 if a bounded wait gave up."""
    rc = _lib().gbnn_status(int(reset))
    if rc < 0:
        raise RuntimeError(f"gbnn_status failed ({rc})")
    return rc


def conv3x3_fwd(x, xs, w, bias, y, ys, N, H, W, cin, cout, relu, mask=None, ms=0, stream=None):
    _ck(_lib().gbnn_conv3x3_fwd(_p(x), xs, _p(w), _p(bias), _p(y), ys, _p(mask), ms, N, H, W, cin, cout, int(relu),
                                _s(stream)), "gbnn_conv3x3_fwd")


def flip_weights(w, wf, cout, cin, stream=None):
    _ck(_lib().gbnn_flip_weights(_p(w), _p(wf), cout, cin, _s(stream)), "gbnn_flip_weights")


def conv3x3_dgrad(gy, gys, wf, gx, gxs, N, H, W, cin, cout, mask=None, ms=0, stream=None):
    _ck(_lib().gbnn_conv3x3_dgrad(_p(gy), gys, _p(wf), _p(gx), gxs, _p(mask), ms, N, H, W, cin, cout, _s(stream)),
        "gbnn_conv3x3_dgrad")


def conv3x3_wgrad(x, xs, gy, gys, gw, gb, N, H, W, cin, cout, splits=0, stream=None):
    _ck(_lib().gbnn_conv3x3_wgrad(_p(x), xs, _p(gy), gys, _p(gw), _p(gb), N, H, W, cin, cout, splits, _s(stream)),
        "gbnn_conv3x3_wgrad")


def avgpool2(x, xs, y, ys, N, H, W, C, stream=None):
    _ck(_lib().gbnn_avgpool2(_p(x), xs, _p(y), ys, N, H, W, C, _s(stream)), "gbnn_avgpool2")


def avgpool2_bwd(gy, gys, gx, gxs, N, H, W, C, accumulate=False, mask=None, ms=0, stream=None):
    _ck(_lib().gbnn_avgpool2_bwd(_p(gy), gys, _p(gx), gxs, _p(mask), ms, N, H, W, C, int(accumulate), _s(stream)),
        "gbnn_avgpool2_bwd")


def upsample2(x, xs, y, ys, N, H, W, C, stream=None):
    _ck(_lib().gbnn_upsample2(_p(x), xs, _p(y), ys, N, H, W, C, _s(stream)), "gbnn_upsample2")


def upsample2_bwd(gy, gys, gx, gxs, N, H, W, C, stream=None):
    _ck(_lib().gbnn_upsample2_bwd(_p(gy), gys, _p(gx), gxs, N, H, W, C, _s(stream)), "gbnn_upsample2_bwd")


def mse(pred, ps, target, weight, grad, gs, P, C, scale, loss_sum, stream=None):
    _ck(_lib().gbnn_mse(_p(pred), ps, _p(target), _p(weight), _p(grad), gs, int(P), C, float(scale), _p(loss_sum),
                        _s(stream)), "gbnn_mse")


def adam(param, grad, m, v, param_bf16, n, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _ck(_lib().gbnn_adam(_p(param), _p(grad), _p(m), _p(v), _p(param_bf16), int(n), float(lr), float(beta1),
                         float(beta2), float(eps), int(t), _s(stream)), "gbnn_adam")


def encode_input(solid, re_feature, phase, H, W, x, stream=None, wave_k=0.0, wave_x0=0.0):
    _ck(_lib().gbnn_encode_input(_p(solid), float(re_feature), float(phase), float(wave_k), float(wave_x0), H, W, _p(x),
                                 _s(stream)), "gbnn_encode_input")


def encode_target(rho, u, v, solid, P, U, vel_scale, rho_scale, target, weight, stream=None):
    _ck(_lib().gbnn_encode_target(_p(rho), _p(u), _p(v), _p(solid), int(P), float(U), float(vel_scale),
                                  float(rho_scale), _p(target), _p(weight), _s(stream)), "gbnn_encode_target")


def decode_output(out, os_, solid, P, U, vel_scale, rho_scale, rho, u, v, stream=None):
    _ck(_lib().gbnn_decode_output(_p(out), os_, _p(solid), int(P), float(U), float(vel_scale), float(rho_scale),
                                  _p(rho), _p(u), _p(v), _s(stream)), "gbnn_decode_output")


def fill_zero(t, stream=None):
    _ck(_lib().gbnn_fill_zero(_p(t), t.numel() * t.element_size(), _s(stream)), "gbnn_fill_zero")


# --------------------------------------------------------------- network


class Conv:
    """One 3x3 convolution: FP32 master weights, bfloat16 copies (forward
    and flipped for the input gradient), FP32 gradients and Adam moments."""

    def __init__(self, cin, cout, rng, device, relu=True, zero=False):
        import torch
        self.cin, self.cout, self.relu = cin, cout, relu
        std = np.sqrt(2.0 / (9 * cin)) if not zero else 0.0
        w = (rng.standard_normal((cout, 3, 3, cin)) * std).astype(np.float32)
        self.w = torch.from_numpy(w).to(device)
        self.b = torch.zeros(cout, dtype=torch.float32, device=device)
        self.w16 = torch.empty((cout, 3, 3, cin), dtype=torch.bfloat16, device=device)
        self.wf16 = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=device)
        self.gw = torch.empty_like(self.w)
        self.gb = torch.empty_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.sync_bf16(None, t=0)

    def sync_bf16(self, stream, t):
        # the bf16 copy is written by the Adam kernel; at t = 0 a zero-rate step makes it
        if t == 0:
            zero_g = self.gw.new_zeros(self.gw.shape)
            adam(self.w, zero_g, self.mw, self.vw, self.w16, self.w.numel(), 0.0, 1, stream=stream)
        flip_weights(self.w16, self.wf16, self.cout, self.cin, stream)

    def zero_grad(self, stream):
        fill_zero(self.gw, stream)
        fill_zero(self.gb, stream)

    def params(self):
        return [(self.w, self.gw, self.mw, self.vw, self.w16), (self.b, self.gb, self.mb, self.vb, None)]


class WarmStartNet:
    """Encoder-decoder 8 -> 32-64-128-256 -> 32 -> 8 (first 3 outputs used)
    on N samples of H x W (both divisible by 8)."""

    IN_C = 8
    OUT_C = 8

    def __init__(self, N, H, W, device, seed=0, zero_head=False):
        import torch
        assert H % 8 == 0 and W % 8 == 0
        self.N, self.H, self.W = N, H, W
        self.device = device
        rng = np.random.default_rng(seed)
        C = [32, 64, 128, 256]
        self.layers = {
            "c1a": Conv(self.IN_C, C[0], rng, device), "c1b": Conv(C[0], C[0], rng, device),
            "c2a": Conv(C[0], C[1], rng, device), "c2b": Conv(C[1], C[1], rng, device),
            "c3a": Conv(C[1], C[2], rng, device), "c3b": Conv(C[2], C[2], rng, device),
            "c4a": Conv(C[2], C[3], rng, device), "c4b": Conv(C[3], C[3], rng, device),
            "d3a": Conv(C[3] + C[2], C[2], rng, device), "d3b": Conv(C[2], C[2], rng, device),
            "d2a": Conv(C[2] + C[1], C[1], rng, device), "d2b": Conv(C[1], C[1], rng, device),
            "d1a": Conv(C[1] + C[0], C[0], rng, device), "d1b": Conv(C[0], C[0], rng, device),
            "head": Conv(C[0], self.OUT_C, rng, device, relu=False, zero=zero_head),
        }
        self.t = 0
        bf = torch.bfloat16

        def act(h, w, c):
            return torch.empty((N, h, w, c), dtype=bf, device=device)

        H1, W1, H2, W2, H3, W3, H4, W4 = H, W, H // 2, W // 2, H // 4, W // 4, H // 8, W // 8
        self.dims = [(H1, W1), (H2, W2), (H3, W3), (H4, W4)]
        self.x0 = act(H1, W1, self.IN_C)
        # forward activations; cat_l holds [upsampled decoder | encoder skip]
        self.a1, self.cat1 = act(H1, W1, 32), act(H1, W1, 96)
        self.p1, self.a2, self.cat2 = act(H2, W2, 32), act(H2, W2, 64), act(H2, W2, 192)
        self.p2, self.a3, self.cat3 = act(H3, W3, 64), act(H3, W3, 128), act(H3, W3, 384)
        self.p3, self.a4, self.b4 = act(H4, W4, 128), act(H4, W4, 256), act(H4, W4, 256)
        self.e3, self.d3 = act(H3, W3, 128), act(H3, W3, 128)
        self.e2, self.d2 = act(H2, W2, 64), act(H2, W2, 64)
        self.e1, self.d1 = act(H1, W1, 32), act(H1, W1, 32)
        self.out = act(H1, W1, self.OUT_C)
        # gradients (w.r.t. pre-activations where a ReLU follows)
        self.g_out = act(H1, W1, self.OUT_C)
        self.g_d1, self.g_e1, self.g_cat1 = act(H1, W1, 32), act(H1, W1, 32), act(H1, W1, 96)
        self.g_d2, self.g_e2, self.g_cat2 = act(H2, W2, 64), act(H2, W2, 64), act(H2, W2, 192)
        self.g_d3, self.g_e3, self.g_cat3 = act(H3, W3, 128), act(H3, W3, 128), act(H3, W3, 384)
        self.g_b4, self.g_a4, self.g_p3 = act(H4, W4, 256), act(H4, W4, 256), act(H4, W4, 128)
        self.g_a3, self.g_p2 = act(H3, W3, 128), act(H3, W3, 64)
        self.g_a2, self.g_p1 = act(H2, W2, 64), act(H2, W2, 32)
        self.g_a1 = act(H1, W1, 32)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    # ------------------------------------------------------------ forward
    def forward(self, stream=None):
        N, L = self.N, self.layers
        (H1, W1), (H2, W2), (H3, W3), (H4, W4) = self.dims

        def conv(name, x, xs, y, ys, h, w):
            c = L[name]
            conv3x3_fwd(x, xs, c.w16, c.b, y, ys, N, h, w, c.cin, c.cout, c.relu, stream=stream)

        conv("c1a", self.x0, 8, self.a1, 32, H1, W1)
        s1 = self.cat1[..., 64:]
        conv("c1b", self.a1, 32, s1, 96, H1, W1)
        avgpool2(s1, 96, self.p1, 32, N, H1, W1, 32, stream)
        conv("c2a", self.p1, 32, self.a2, 64, H2, W2)
        s2 = self.cat2[..., 128:]
        conv("c2b", self.a2, 64, s2, 192, H2, W2)
        avgpool2(s2, 192, self.p2, 64, N, H2, W2, 64, stream)
        conv("c3a", self.p2, 64, self.a3, 128, H3, W3)
        s3 = self.cat3[..., 256:]
        conv("c3b", self.a3, 128, s3, 384, H3, W3)
        avgpool2(s3, 384, self.p3, 128, N, H3, W3, 128, stream)
        conv("c4a", self.p3, 128, self.a4, 256, H4, W4)
        conv("c4b", self.a4, 256, self.b4, 256, H4, W4)
        upsample2(self.b4, 256, self.cat3, 384, N, H4, W4, 256, stream)
        conv("d3a", self.cat3, 384, self.e3, 128, H3, W3)
        conv("d3b", self.e3, 128, self.d3, 128, H3, W3)
        upsample2(self.d3, 128, self.cat2, 192, N, H3, W3, 128, stream)
        conv("d2a", self.cat2, 192, self.e2, 64, H2, W2)
        conv("d2b", self.e2, 64, self.d2, 64, H2, W2)
        upsample2(self.d2, 64, self.cat1, 96, N, H2, W2, 64, stream)
        conv("d1a", self.cat1, 96, self.e1, 32, H1, W1)
        conv("d1b", self.e1, 32, self.d1, 32, H1, W1)
        conv("head", self.d1, 32, self.out, self.OUT_C, H1, W1)
        return self.out

    # ------------------------------------------------------------ backward
    def backward(self, stream=None):
        """Gradients of all parameters given self.g_out = dL/d(out)."""
        N, L = self.N, self.layers
        (H1, W1), (H2, W2), (H3, W3), (H4, W4) = self.dims
        for c in L.values():
            c.zero_grad(stream)

        def wgrad(name, x, xs, gy, gys, h, w):
            c = L[name]
            conv3x3_wgrad(x, xs, gy, gys, c.gw, c.gb, N, h, w, c.cin, c.cout, stream=stream)

        def dgrad(name, gy, gys, gx, gxs, h, w, mask=None, ms=0):
            c = L[name]
            conv3x3_dgrad(gy, gys, c.wf16, gx, gxs, N, h, w, c.cin, c.cout, mask=mask, ms=ms, stream=stream)

        # head (no activation): d1 = relu output -> mask by d1
        wgrad("head", self.d1, 32, self.g_out, self.OUT_C, H1, W1)
        dgrad("head", self.g_out, self.OUT_C, self.g_d1, 32, H1, W1, self.d1, 32)
        wgrad("d1b", self.e1, 32, self.g_d1, 32, H1, W1)
        dgrad("d1b", self.g_d1, 32, self.g_e1, 32, H1, W1, self.e1, 32)
        wgrad("d1a", self.cat1, 96, self.g_e1, 32, H1, W1)
        dgrad("d1a", self.g_e1, 32, self.g_cat1, 96, H1, W1, self.cat1, 96)
        # decoder path up to level 2: upsample backward of the d2 part
        upsample2_bwd(self.g_cat1, 96, self.g_d2, 64, N, H2, W2, 64, stream)
        wgrad("d2b", self.e2, 64, self.g_d2, 64, H2, W2)
        dgrad("d2b", self.g_d2, 64, self.g_e2, 64, H2, W2, self.e2, 64)
        wgrad("d2a", self.cat2, 192, self.g_e2, 64, H2, W2)
        dgrad("d2a", self.g_e2, 64, self.g_cat2, 192, H2, W2, self.cat2, 192)
        upsample2_bwd(self.g_cat2, 192, self.g_d3, 128, N, H3, W3, 128, stream)
        wgrad("d3b", self.e3, 128, self.g_d3, 128, H3, W3)
        dgrad("d3b", self.g_d3, 128, self.g_e3, 128, H3, W3, self.e3, 128)
        wgrad("d3a", self.cat3, 384, self.g_e3, 128, H3, W3)
        dgrad("d3a", self.g_e3, 128, self.g_cat3, 384, H3, W3, self.cat3, 384)
        upsample2_bwd(self.g_cat3, 384, self.g_b4, 256, N, H4, W4, 256, stream)
        # bottom
        wgrad("c4b", self.a4, 256, self.g_b4, 256, H4, W4)
        dgrad("c4b", self.g_b4, 256, self.g_a4, 256, H4, W4, self.a4, 256)
        wgrad("c4a", self.p3, 128, self.g_a4, 256, H4, W4)
        dgrad("c4a", self.g_a4, 256, self.g_p3, 128, H4, W4)
        # encoder level 3: skip gradient (already masked) + pooled path (masked by s3)
        g_s3 = self.g_cat3[..., 256:]
        avgpool2_bwd(self.g_p3, 128, g_s3, 384, N, H3, W3, 128, accumulate=True, mask=self.cat3[..., 256:], ms=384,
                     stream=stream)
        wgrad("c3b", self.a3, 128, g_s3, 384, H3, W3)
        dgrad("c3b", g_s3, 384, self.g_a3, 128, H3, W3, self.a3, 128)
        wgrad("c3a", self.p2, 64, self.g_a3, 128, H3, W3)
        dgrad("c3a", self.g_a3, 128, self.g_p2, 64, H3, W3)
        g_s2 = self.g_cat2[..., 128:]
        avgpool2_bwd(self.g_p2, 64, g_s2, 192, N, H2, W2, 64, accumulate=True, mask=self.cat2[..., 128:], ms=192,
                     stream=stream)
        wgrad("c2b", self.a2, 64, g_s2, 192, H2, W2)
        dgrad("c2b", g_s2, 192, self.g_a2, 64, H2, W2, self.a2, 64)
        wgrad("c2a", self.p1, 32, self.g_a2, 64, H2, W2)
        dgrad("c2a", self.g_a2, 64, self.g_p1, 32, H2, W2)
        g_s1 = self.g_cat1[..., 64:]
        avgpool2_bwd(self.g_p1, 32, g_s1, 96, N, H1, W1, 32, accumulate=True, mask=self.cat1[..., 64:], ms=96,
                     stream=stream)
        wgrad("c1b", self.a1, 32, g_s1, 96, H1, W1)
        dgrad("c1b", g_s1, 96, self.g_a1, 32, H1, W1, self.a1, 32)
        wgrad("c1a", self.x0, 8, self.g_a1, 32, H1, W1)

    def adam_step(self, lr, stream=None):
        self.t += 1
        for c in self.layers.values():
            for (p, g, m, v, p16) in c.params():
                adam(p, g, m, v, p16, p.numel(), lr, self.t, stream=stream)
            flip_weights(c.w16, c.wf16, c.cout, c.cin, stream)

    def loss_and_grad(self, target, weight, stream=None):
        """MSE over the first 3 output channels of fluid pixels; fills g_out."""
        P = self.N * self.H * self.W
        fill_zero(self.g_out, stream)
        fill_zero(self.loss, stream)
        mse(self.out, self.OUT_C, target, weight, self.g_out, self.OUT_C, P, 3, 1.0 / (3 * P), self.loss, stream)
        return self.loss

    def state(self) -> dict:
        """Host copy of the FP32 master weights and biases (name -> array)."""
        out = {}
        for name, c in self.layers.items():
            out[name + ".w"] = c.w.detach().cpu().numpy()
            out[name + ".b"] = c.b.detach().cpu().numpy()
        return out

    def load_state(self, st: dict, stream=None):
        """Set the weights from `state()` output and refresh the bfloat16 copies."""
        import torch
        for name, c in self.layers.items():
            c.w.copy_(torch.from_numpy(np.ascontiguousarray(st[name + ".w"])))
            c.b.copy_(torch.from_numpy(np.ascontiguousarray(st[name + ".b"])))
            c.sync_bf16(stream, t=0)

    def flops_per_sample(self) -> float:
        """Multiply-adds x 2 of the forward convolutions of one sample."""
        tot = 0.0
        sizes = {"c1": 0, "d1": 0, "he": 0, "c2": 1, "d2": 1, "c3": 2, "d3": 2, "c4": 3}
        for name, c in self.layers.items():
            h, w = self.dims[sizes[name[:2]]]
            tot += 2.0 * h * w * 9 * c.cin * c.cout
        return tot
