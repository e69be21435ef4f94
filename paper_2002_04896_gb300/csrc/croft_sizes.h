// croft_sizes.h - every supported axis length 2 <= n <= 4096 of the form 2^a 3^b 5^c,
// split into four interleaved groups so the kernel instantiations compile in parallel.
#pragma once

#define CROFT_SIZES_0(X) X(2) X(6) X(12) X(20) X(30) X(45) X(60) X(80) X(100) X(128) X(160) X(200) X(243) \
    X(288) X(360) X(405) X(486) X(576) X(648) X(750) X(864) X(1000) X(1152) X(1280) X(1458) X(1620) X(1920) \
    X(2048) X(2304) X(2560) X(2916) X(3200) X(3600) X(3888)

#define CROFT_SIZES_1(X) X(3) X(8) X(15) X(24) X(32) X(48) X(64) X(81) X(108) X(135) X(162) X(216) X(250) \
    X(300) X(375) X(432) X(500) X(600) X(675) X(768) X(900) X(1024) X(1200) X(1296) X(1500) X(1728) X(1944) \
    X(2160) X(2400) X(2592) X(3000) X(3240) X(3645) X(4000)

#define CROFT_SIZES_2(X) X(4) X(9) X(16) X(25) X(36) X(50) X(72) X(90) X(120) X(144) X(180) X(225) X(256) \
    X(320) X(384) X(450) X(512) X(625) X(720) X(800) X(960) X(1080) X(1215) X(1350) X(1536) X(1800) X(2000) \
    X(2187) X(2430) X(2700) X(3072) X(3375) X(3750) X(4050)

#define CROFT_SIZES_3(X) X(5) X(10) X(18) X(27) X(40) X(54) X(75) X(96) X(125) X(150) X(192) X(240) X(270) \
    X(324) X(400) X(480) X(540) X(640) X(729) X(810) X(972) X(1125) X(1250) X(1440) X(1600) X(1875) X(2025) \
    X(2250) X(2500) X(2880) X(3125) X(3456) X(3840) X(4096)

// complex128 lengths (croft_kernels64.cu, croft_conv.cu): every power of two up to
// 1024 and a few mixed-radix ones.
#define CROFT_SIZES64(X) \
    X(2) X(3) X(4) X(5) X(6) X(8) X(10) X(12) X(15) X(16) X(32) X(48) X(60) X(64) X(96) X(120) X(128) X(256) X(512) X(1024)

// Batched plans: every axis length <= 128 of the form 2^a 3^b 5^c (the per-system PME
// mesh range; croft_batched.cu, croft_batch_group.cu).
#define CROFT_BATCH_SIZES(X)                                                                                \
    X(2) X(3) X(4) X(5) X(6) X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32)     \
    X(36) X(40) X(45) X(48) X(50) X(54) X(60) X(64) X(72) X(75) X(80) X(81) X(90) X(96) X(100) X(108)       \
    X(120) X(125) X(128)
