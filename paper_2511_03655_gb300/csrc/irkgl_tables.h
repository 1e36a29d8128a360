/* Generated by paper_2511_03655_gb300/gen_tables.py -- do not edit.
 * IRKGL16 FP64 tables (arXiv 2511.03655 Sec. 2.2-2.4), row-major [i*8+j]:
 * c, b: nodes and weights; MU (Eq. Yi2); ETA (Eq. Qi2, Eq. sympl_cond_2 exact);
 * NU (Eq. Pol0, scaled by 1/b); W = A nut diag(1/b) (fused initial guess). */
#pragma once

static const double IRKGL_TAB_C[8] = {
  0x1.454e34f533998p-6,
  0x1.a06d536d82f88p-4,
  0x1.e5dad4f9af698p-3,
  0x1.a214dac30e32fp-2,
  0x1.2ef5929e78e69p-1,
  0x1.86894ac19425ap-1,
  0x1.cbf255924fa0fp-1,
  0x1.f5d58e5856633p-1};

static const double IRKGL_TAB_B[8] = {
  0x1.9ea1d04ca0374p-5,
  0x1.c76fb531d2b96p-4,
  0x1.413c50a255615p-3,
  0x1.736360b199343p-3,
  0x1.736360b199343p-3,
  0x1.413c50a255615p-3,
  0x1.c76fb531d2b96p-4,
  0x1.9ea1d04ca0374p-5};

static const double IRKGL_TAB_MU[64] = {
  0x1.0000000000000p-1, -0x1.4f7117c3edf90p-4, 0x1.4807a2e56e190p-5, -0x1.9508d6ef38f80p-6, 0x1.16233b3721e80p-6, -0x1.909e66a3e1880p-7, 0x1.1eac4c148db80p-7, -0x1.6752422346f00p-8,
  0x1.14f7117c3edf9p+0, 0x1.0000000000000p-1, -0x1.642f0a7f7a890p-4, 0x1.70285f76e2c70p-5, -0x1.d7333dc6adb00p-6, 0x1.47f5eb23ba180p-6, -0x1.cd304120cc600p-7, 0x1.1eac4c148db80p-7,
  0x1.eb7f85d1a91e7p-1, 0x1.1642f0a7f7a89p+0, 0x1.0000000000000p-1, -0x1.68d515c5598c0p-4, 0x1.7a2fff32b1ce0p-5, -0x1.e507a4a989780p-6, 0x1.47f5eb23ba180p-6, -0x1.909e66a3e1880p-7,
  0x1.0654235bbce3ep+0, 0x1.e8fd7a0891d39p-1, 0x1.168d515c5598cp+0, 0x1.0000000000000p-1, -0x1.69deb67a94160p-4, 0x1.7a2fff32b1ce0p-5, -0x1.d7333dc6adb00p-6, 0x1.16233b3721e80p-6,
  0x1.f74ee62646f0cp-1, 0x1.075cccf71ab6cp+0, 0x1.e85d000cd4e32p-1, 0x1.169deb67a9416p+0, 0x1.0000000000000p-1, -0x1.68d515c5598c0p-4, 0x1.70285f76e2c70p-5, -0x1.9508d6ef38f80p-6,
  0x1.03213ccd47c31p+0, 0x1.f5c050a6e22f4p-1, 0x1.07941e92a625ep+0, 0x1.e85d000cd4e32p-1, 0x1.168d515c5598cp+0, 0x1.0000000000000p-1, -0x1.642f0a7f7a890p-4, 0x1.4807a2e56e190p-5,
  0x1.fb854ecfadc92p-1, 0x1.039a60824198cp+0, 0x1.f5c050a6e22f4p-1, 0x1.075cccf71ab6cp+0, 0x1.e8fd7a0891d39p-1, 0x1.1642f0a7f7a89p+0, 0x1.0000000000000p-1, -0x1.4f7117c3edf90p-4,
  0x1.016752422346fp+0, 0x1.fb854ecfadc92p-1, 0x1.03213ccd47c31p+0, 0x1.f74ee62646f0cp-1, 0x1.0654235bbce3ep+0, 0x1.eb7f85d1a91e7p-1, 0x1.14f7117c3edf9p+0, 0x1.0000000000000p-1};

static const double IRKGL_TAB_ETA[64] = {
  0x1.89b89dc278c8dp-8, -0x1.10c068fb3b100p-9, 0x1.be2ad5836b380p-10, -0x1.9e4b7384dd180p-10, 0x1.829e22d996380p-10, -0x1.5afd24848ee80p-10, 0x1.1f2bbee8f4780p-10, -0x1.855929d082900p-11,
  0x1.4693c2e85c39ap-4, 0x1.a48d0e3ca1b40p-7, -0x1.c0705b64661c0p-9, 0x1.503bd909c6000p-9, -0x1.2711178341380p-9, 0x1.03195a19dd600p-9, -0x1.a919c68ba0400p-10, 0x1.1f2bbee8f4800p-10,
  0x1.c0ad64060fcccp-3, 0x1.0ea269d55c54dp-3, 0x1.2755a462d62b5p-6, -0x1.19f5b4a38e380p-8, 0x1.89fa9d4c31700p-9, -0x1.437c2bc003800p-9, 0x1.03195a19dd600p-9, -0x1.5afd24848ee00p-10,
  0x1.8c21ac00361c4p-2, 0x1.3c99fd99c100dp-2, 0x1.557f32e7508aap-3, 0x1.550c99ba93970p-6, -0x1.2e2003ef48d80p-8, 0x1.89fa9d4c31780p-9, -0x1.2711178341300p-9, 0x1.829e22d996500p-10,
  0x1.258c70083c14ep-1, 0x1.f381ae328a8c9p-2, 0x1.6e11affab27b4p-2, 0x1.6e3b94d44cedap-3, 0x1.550c99ba93970p-6, -0x1.19f5b4a38e340p-8, 0x1.503bd909c6080p-9, -0x1.9e4b7384dd000p-10,
  0x1.7bb15a87a8416p-1, 0x1.537eb9adfda3fp-1, 0x1.0bcf19576847cp-1, 0x1.6e11affab27b4p-2, 0x1.557f32e7508aap-3, 0x1.2755a462d62b5p-6, -0x1.c0705b64661c0p-9, 0x1.be2ad5836b400p-10,
  0x1.c25779ca1a7e6p-1, 0x1.97101e415971cp-1, 0x1.537eb9adfda3fp-1, 0x1.f381ae328a8c9p-2, 0x1.3c99fd99c100dp-2, 0x1.0ea269d55c54dp-3, 0x1.a48d0e3ca1b40p-7, -0x1.10c068fb3b0c0p-9,
  0x1.eb49c66638a5cp-1, 0x1.c25779ca1a7e6p-1, 0x1.7bb15a87a8416p-1, 0x1.258c70083c14ep-1, 0x1.8c21ac00361c4p-2, 0x1.c0ad64060fcccp-3, 0x1.4693c2e85c39ap-4, 0x1.89b89dc278c8dp-8};

static const double IRKGL_TAB_NU[64] = {
  -0x1.82578299ae8e1p-6, 0x1.33b97a149941fp-5, -0x1.ac898c9579e0ap-5, 0x1.2789efe540dcep-4, -0x1.a8ab48c9127d2p-4, 0x1.4d7d24c5f3cb6p-3, -0x1.3598c693b9092p-2, 0x1.8932d606bd4e5p-1,
  -0x1.7974c9f44f16bp-1, 0x1.2b18f474d3161p+0, -0x1.9c06828f5944bp+0, 0x1.16738b3c41e9bp+1, -0x1.80f36d71f5b70p+1, 0x1.16be7a2387c5cp+2, -0x1.a7752b0ac86f2p+2, 0x1.25f3e8706ae28p+3,
  -0x1.8986c2c12c30fp+3, 0x1.35578de3cd220p+4, -0x1.a329da490e726p+4, 0x1.13010d1cfa812p+5, -0x1.68ab75a434d50p+5, 0x1.d9f91454f1d2fp+5, -0x1.2b17072ad4e46p+6, 0x1.2ae212444cf84p+6,
  -0x1.ee6bb76ec6117p+6, 0x1.816c9774d8e44p+7, -0x1.00c9832ed4955p+8, 0x1.476150b7858e8p+8, -0x1.9973c2ef6d093p+8, 0x1.f233812fe14c5p+8, -0x1.1742225b33835p+9, 0x1.e130205dba74fp+8,
  -0x1.7e882400ddbebp+9, 0x1.281455735a453p+10, -0x1.850672850953dp+10, 0x1.e49ce7b9f0c70p+10, -0x1.2463fa668632cp+11, 0x1.518fe7993d1e3p+11, -0x1.6105d9813da83p+11, 0x1.1b89cfd1cf5a0p+11,
  -0x1.754efb0741a04p+11, 0x1.1f62783291843p+12, -0x1.75af950c42931p+12, 0x1.c9cde4a219d96p+12, -0x1.0d830ff6f1095p+13, 0x1.2ce00c0e553f9p+13, -0x1.2e3a51501d4a2p+13, 0x1.d45e9421158f4p+12,
  -0x1.d6c418ae96257p+12, 0x1.6919f48834114p+13, -0x1.d2501238d6f62p+13, 0x1.1a92a13c823dep+14, -0x1.479f2af354809p+14, 0x1.6678ace869e3bp+14, -0x1.5ffee8001d9a4p+14, 0x1.0ba7abbc13d0dp+14,
  -0x1.870ed3f67fa80p+13, 0x1.2b6042908a79fp+14, -0x1.812d94aa4f86bp+14, 0x1.d0288568ab926p+14, -0x1.0af0a862e5235p+15, 0x1.2121122e8fc3dp+15, -0x1.18c6a44733fe7p+15, 0x1.a73b38b217a66p+14};

static const double IRKGL_TAB_W[64] = {
  0x1.f0b4351b27ec3p-12, -0x1.5d9550d41c71dp-11, 0x1.7c8989f6f1006p-11, -0x1.53be680ef30f1p-11, 0x1.94ad08b296c53p-12, 0x1.9de49d9371c18p-13, -0x1.9f113614f4f76p-10, 0x1.a62d54726655bp-8,
  -0x1.6c9d63f8c83b4p-6, 0x1.205ac58592d7ep-5, -0x1.8c2f9612fe8a7p-5, 0x1.0b59f31b668e6p-4, -0x1.72c4890ac17cep-4, 0x1.10a0c4ecb7298p-3, -0x1.b29c010ebb26ap-3, 0x1.5d35860e774a2p-2,
  -0x1.46e4891c74bb7p-1, 0x1.01a7ca0185d12p+0, -0x1.5f0b947f8ac49p+0, 0x1.d11c56a6730c3p+0, -0x1.36355712e85b2p+1, 0x1.a45f27ba7f38cp+1, -0x1.19166870d180cp+2, 0x1.382708cc97fb4p+2,
  -0x1.2d6fc7419cd7dp+3, 0x1.d773515837a48p+3, -0x1.3c19364c7a55ap+4, 0x1.976afb2b9a031p+4, -0x1.036c74c4830ffp+5, 0x1.4524b12a294fbp+5, -0x1.7dfaaeb4c4d27p+5, 0x1.5e8acfd79fe76p+5,
  -0x1.319da521ad63ap+6, 0x1.dab520a919997p+6, -0x1.39f7b6fb26a69p+7, 0x1.8b82bf78ff445p+7, -0x1.e5b29d3c9b971p+7, 0x1.1fd9dc86474a8p+8, -0x1.383a1d2b649aap+8, 0x1.05102534acc8ap+8,
  -0x1.6928be24395d9p+8, 0x1.16ff2b6a9a8b0p+9, -0x1.6d3b2b3de5d23p+9, 0x1.c45c1429220b5p+9, -0x1.0eb84dad631fap+10, 0x1.355661768e213p+10, -0x1.400bbf04e293bp+10, 0x1.fe73d3b8cc8f9p+9,
  -0x1.02662d2ddb281p+10, 0x1.8dc7dd6b4f9c0p+10, -0x1.028d024d7a0b2p+11, 0x1.3caeb8bdb5a39p+11, -0x1.74e8379bfa925p+11, 0x1.a0bac4825b584p+11, -0x1.a3bdbc011eec7p+11, 0x1.469d10191b494p+11,
  -0x1.cbad7a3915b12p+10, 0x1.611da5b7c1f4dp+11, -0x1.c94ef60ad3632p+11, 0x1.1667ea7b6b687p+12, -0x1.450cd13829414p+12, 0x1.672ae1d6a8887p+12, -0x1.650bd77a2c0bdp+12, 0x1.12abc624c6e98p+12};

// s-stage variants (s = 2, 4, 6) for the first-order form: c, b [s]; MU, NU
// [s*s], row-major [i*s+j], built by the same route as the 8-stage tables.
static const double IRKGL_TAB2_C[2] = {
  0x1.b0cb174df99c7p-3,
  0x1.93cd3a2c8198ep-1};

static const double IRKGL_TAB2_B[2] = {
  0x1.0000000000000p-1,
  0x1.0000000000000p-1};

static const double IRKGL_TAB2_MU[4] = {
  0x1.0000000000000p-1,
  -0x1.3cd3a2c8198e0p-4,
  0x1.13cd3a2c8198ep+0,
  0x1.0000000000000p-1};

static const double IRKGL_TAB2_NU[4] = {
  -0x1.db3d742c26554p-3,
  0x1.4f34e8b206639p-1,
  -0x1.a79a74590331cp+0,
  0x1.9db3d742c2655p+1};

static const double IRKGL_TAB4_C[4] = {
  0x1.1c6490c2719ecp-4,
  0x1.51ee013116102p-2,
  0x1.5708ff6774f7fp-1,
  0x1.dc736de7b1cc3p-1};

static const double IRKGL_TAB4_B[4] = {
  0x1.64340f7e7b66bp-3,
  0x1.4de5f840c24cap-2,
  0x1.4de5f840c24cap-2,
  0x1.64340f7e7b66bp-3};

static const double IRKGL_TAB4_MU[16] = {
  0x1.0000000000000p-1,
  -0x1.4e310dc13d440p-4,
  0x1.3d3e2783b9470p-5,
  -0x1.4ee55696af180p-6,
  0x1.14e310dc13d44p+0,
  0x1.0000000000000p-1,
  -0x1.5e392e7fe55a0p-4,
  0x1.3d3e2783b9470p-5,
  0x1.ec2c1d87c46b9p-1,
  0x1.15e392e7fe55ap+0,
  0x1.0000000000000p-1,
  -0x1.4e310dc13d440p-4,
  0x1.053b955a5abc6p+0,
  0x1.ec2c1d87c46b9p-1,
  0x1.14e310dc13d44p+0,
  0x1.0000000000000p-1};

static const double IRKGL_TAB4_NU[16] = {
  -0x1.4a84288582498p-4,
  0x1.314271b529d66p-3,
  -0x1.2543687563367p-2,
  0x1.79883eeedbab0p-1,
  -0x1.9072162b9cf46p+0,
  0x1.5de622def61efp+1,
  -0x1.1d03916fd86f1p+2,
  0x1.abe3b985d97a1p+2,
  -0x1.3e374ac20fe51p+3,
  0x1.084a34312cb12p+4,
  -0x1.7bac264953badp+4,
  0x1.b50e95ee5d666p+4,
  -0x1.a3b0ff8388e07p+4,
  0x1.5321e6da14133p+5,
  -0x1.ca8d4a6579c15p+5,
  0x1.dc880d2a560d9p+5};

static const double IRKGL_TAB6_C[6] = {
  0x1.149ad8bfaff12p-5,
  0x1.5aebed3546d43p-3,
  0x1.85d3b4bf2628fp-2,
  0x1.3d1625a06ceb9p-1,
  0x1.a94504b2ae4afp-1,
  0x1.eeb652740500fp-1};

static const double IRKGL_TAB6_B[6] = {
  0x1.5edf601e2dbf8p-4,
  0x1.716b7b5794c1cp-3,
  0x1.df24d499545e8p-3,
  0x1.df24d499545e8p-3,
  0x1.716b7b5794c1cp-3,
  0x1.5edf601e2dbf8p-4};

static const double IRKGL_TAB6_MU[36] = {
  0x1.0000000000000p-1,
  -0x1.4f3f613ad9440p-4,
  0x1.46843ad297020p-5,
  -0x1.8cfd6eea15380p-6,
  0x1.0344b4f645be0p-6,
  -0x1.36e8c17fada80p-7,
  0x1.14f3f613ad944p+0,
  0x1.0000000000000p-1,
  -0x1.63676619522a0p-4,
  0x1.6adda35673db0p-5,
  -0x1.bbe77274b3f80p-6,
  0x1.0344b4f645be0p-6,
  0x1.eb97bc52d68fep-1,
  0x1.163676619522ap+0,
  0x1.0000000000000p-1,
  -0x1.669903c9188a0p-4,
  0x1.6adda35673db0p-5,
  -0x1.8cfd6eea15380p-6,
  0x1.0633f5bba854ep+0,
  0x1.e95225ca98c25p-1,
  0x1.1669903c9188ap+0,
  0x1.0000000000000p-1,
  -0x1.63676619522a0p-4,
  0x1.46843ad297020p-5,
  0x1.f7e5da584dd21p-1,
  0x1.06ef9dc9d2cfep+0,
  0x1.e95225ca98c25p-1,
  0x1.163676619522ap+0,
  0x1.0000000000000p-1,
  -0x1.4f3f613ad9440p-4,
  0x1.026dd182ff5b5p+0,
  0x1.f7e5da584dd21p-1,
  0x1.0633f5bba854ep+0,
  0x1.eb97bc52d68fep-1,
  0x1.14f3f613ad944p+0,
  0x1.0000000000000p-1};

static const double IRKGL_TAB6_NU[36] = {
  -0x1.467af1809201ap-5,
  0x1.0ee173acd427bp-4,
  -0x1.99b87b1479ebbp-4,
  0x1.470763eae03eap-3,
  -0x1.311e1273602f7p-2,
  0x1.84bfddeb7a100p-1,
  -0x1.14151cdb54a95p+0,
  0x1.c39816597115ep+0,
  -0x1.4a450857906ffp+1,
  0x1.e9109b949a170p+1,
  -0x1.79068404d8fdbp+2,
  0x1.0b746ecb4c0fcp+3,
  -0x1.a157963daf826p+3,
  0x1.4eebc7703330bp+4,
  -0x1.d5c93cea80dfbp+4,
  0x1.3fdc5d37d20c4p+5,
  -0x1.a0fb92a1d6c7dp+5,
  0x1.b1408caa6cd45p+5,
  -0x1.4523a588af22ep+6,
  0x1.00bcaaf5e45a2p+7,
  -0x1.5c18b17988491p+7,
  0x1.bdd19a24ed17cp+7,
  -0x1.066bf9248b590p+8,
  0x1.dab112ea1851bp+7,
  -0x1.1482525dda0bbp+8,
  0x1.afe1ef469936bp+8,
  -0x1.1e573c76410fep+9,
  0x1.6144fa039d0b4p+9,
  -0x1.898c2f9a432f9p+9,
  0x1.4e4ca39315f56p+9,
  -0x1.0cbb0b8b36816p+9,
  0x1.a144dcb4ebd79p+9,
  -0x1.1176bbf2eda8ap+10,
  0x1.4b24e9cee0afdp+10,
  -0x1.677fee84612cap+10,
  0x1.2954c75d3fd8bp+10};

// Explicit splitting baselines (Sec. 4, Eq. high_order_splitting): drift weights a[s+1],
// kick weights b[s]; Strang (s = 1) and Suzuki's fourth-order composition (s = 5).
static const double IRKGL_SPLIT_STRANG_A[2] = {
  0x1.0000000000000p-1,
  0x1.0000000000000p-1};

static const double IRKGL_SPLIT_STRANG_B[1] = {
  0x1.0000000000000p+0};

static const double IRKGL_SPLIT_SUZ90_A[6] = {
  0x1.a87044d5670efp-3,
  0x1.a87044d5670efp-2,
  -0x1.f2a19d006a59dp-4,
  -0x1.f2a19d006a59dp-4,
  0x1.a87044d5670efp-2,
  0x1.a87044d5670efp-3};

static const double IRKGL_SPLIT_SUZ90_B[5] = {
  0x1.a87044d5670efp-2,
  0x1.a87044d5670efp-2,
  -0x1.50e089aace1dfp-1,
  0x1.a87044d5670efp-2,
  0x1.a87044d5670efp-2};

// Integer forms for the fixed-point mixing (see gen_tables.int_tables):
// |ETA_ij| * 2^63 (exact), round(|W_ij| * 2^50); signs; per-row
// corrections sum_j (+-m_ij) 2^61 as 128-bit two's complement words;
// |MU_ij| * 2^62 (exact) and round(|NU_ij| * 2^47) for the first-order form.
#define IRKGL_ETA_SHIFT 63
#define IRKGL_W_SHIFT 50
#define IRKGL_MU_SHIFT 62
#define IRKGL_NU_SHIFT 47
#define IRKGL_R_BIAS 61
__host__ __device__ constexpr unsigned long long irkgl_eta_mag(int k) {
  constexpr unsigned long long t[64] = {
    0x00c4dc4ee13c6468ull, 0x0044301a3ecec400ull, 0x0037c55ab06d6700ull, 0x0033c96e709ba300ull, 0x003053c45b32c700ull, 0x002b5fa49091dd00ull, 0x0023e577dd1e8f00ull, 0x001855929d082900ull,
    0x0a349e1742e1cd00ull, 0x01a48d0e3ca1b400ull, 0x00701c16d9198700ull, 0x00540ef642718000ull, 0x0049c445e0d04e00ull, 0x0040c65686775800ull, 0x00352338d1740800ull, 0x0023e577dd1e9000ull,
    0x1c0ad64060fccc00ull, 0x10ea269d55c54d00ull, 0x024eab48c5ac56a0ull, 0x008cfada51c71c00ull, 0x00627ea7530c5c00ull, 0x0050df0af000e000ull, 0x0040c65686775800ull, 0x002b5fa49091dc00ull,
    0x3184358006c38800ull, 0x27933fb338201a00ull, 0x1557f32e7508aa00ull, 0x02aa193375272e00ull, 0x00971001f7a46c00ull, 0x00627ea7530c5e00ull, 0x0049c445e0d04c00ull, 0x003053c45b32ca00ull,
    0x49631c020f053800ull, 0x3e7035c651519200ull, 0x2dc235ff564f6800ull, 0x16e3b94d44ceda00ull, 0x02aa193375272e00ull, 0x008cfada51c71a00ull, 0x00540ef642718200ull, 0x0033c96e709ba000ull,
    0x5eec56a1ea105800ull, 0x54dfae6b7f68fc00ull, 0x42f3c655da11f000ull, 0x2dc235ff564f6800ull, 0x1557f32e7508aa00ull, 0x024eab48c5ac56a0ull, 0x00701c16d9198700ull, 0x0037c55ab06d6800ull,
    0x7095de72869f9800ull, 0x65c40790565c7000ull, 0x54dfae6b7f68fc00ull, 0x3e7035c651519200ull, 0x27933fb338201a00ull, 0x10ea269d55c54d00ull, 0x01a48d0e3ca1b400ull, 0x0044301a3ecec300ull,
    0x7ad271998e297000ull, 0x7095de72869f9800ull, 0x5eec56a1ea105800ull, 0x49631c020f053800ull, 0x3184358006c38800ull, 0x1c0ad64060fccc00ull, 0x0a349e1742e1cd00ull, 0x00c4dc4ee13c6468ull};
  return t[k];
}
__host__ __device__ constexpr bool irkgl_eta_neg(int k) { return (0x008040a050a854aaull >> k) & 1ull; }
__host__ __device__ constexpr unsigned irkgl_eta_bias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x00000000u, 0xbd9ed68du, 0x0012a584u,
    0x00000000u, 0x00000000u, 0x9345a180u, 0x01745c4au,
    0x00000000u, 0x00000000u, 0x50730974u, 0x05dbb673u,
    0x00000000u, 0x00000000u, 0x1fdbbd40u, 0x0e196ff7u,
    0x00000000u, 0x00000000u, 0xbe156040u, 0x19d6d49eu,
    0x00000000u, 0x00000000u, 0xb57c71b4u, 0x277e0923u,
    0x00000000u, 0x00000000u, 0x272dddc0u, 0x3470f1afu,
    0x00000000u, 0x00000000u, 0xd337a3adu, 0x3d88091au};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned irkgl_eta_rbias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x00000000u, 0x9aa3438du, 0x00ce5444u,
    0x00000000u, 0x00000000u, 0x1ea37e80u, 0x02635fe0u,
    0x00000000u, 0x00000000u, 0x22cce174u, 0x06e4effdu,
    0x00000000u, 0x00000000u, 0xf8507540u, 0x0efa443eu,
    0x00000000u, 0x00000000u, 0x80781a40u, 0x1a9798e7u,
    0x00000000u, 0x00000000u, 0x8e95f8b4u, 0x27ee253au,
    0x00000000u, 0x00000000u, 0x65fca0c0u, 0x34b521c9u,
    0x00000000u, 0x00000000u, 0xd337a3adu, 0x3d88091au};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned long long irkgl_w_mag(int k) {
  constexpr unsigned long long t[64] = {
    0x0000007c2d0d46caull, 0x000000aecaa86a0eull, 0x000000be44c4fb79ull, 0x000000a9df34077aull, 0x000000652b422ca6ull, 0x00000033bc93b26eull, 0x0000019f113614f5ull, 0x00000698b551c999ull,
    0x000016c9d63f8c84ull, 0x0000240b58b0b25bull, 0x00003185f2c25fd1ull, 0x000042d67cc6d9a4ull, 0x00005cb12242b05full, 0x0000885062765b95ull, 0x0000d94e00875d93ull, 0x00015d35860e774aull,
    0x00028dc91238e977ull, 0x0004069f28061744ull, 0x00057c2e51fe2b12ull, 0x000744715a99cc31ull, 0x0009b1aab89742d9ull, 0x000d22f93dd3f9c6ull, 0x00119166870d180cull, 0x001382708cc97fb4ull,
    0x0025adf8e8339afaull, 0x003aee6a2b06f490ull, 0x004f064d931e9568ull, 0x0065dabecae680c4ull, 0x0081b63a624187f8ull, 0x00a292589514a7d8ull, 0x00befd575a626938ull, 0x00af4567ebcff3b0ull,
    0x01319da521ad63a0ull, 0x01dab520a9199970ull, 0x0273ef6df64d4d20ull, 0x0317057ef1fe88a0ull, 0x03cb653a79372e20ull, 0x047f6772191d2a00ull, 0x04e0e874ad926a80ull, 0x04144094d2b32280ull,
    0x05a4a2f890e57640ull, 0x08b7f95b54d45800ull, 0x0b69d959ef2e9180ull, 0x0e22e0a149105a80ull, 0x10eb84dad631fa00ull, 0x1355661768e21300ull, 0x1400bbf04e293b00ull, 0x0ff39e9dc6647c80ull,
    0x102662d2ddb28100ull, 0x18dc7dd6b4f9c000ull, 0x2051a049af416400ull, 0x2795d717b6b47200ull, 0x2e9d06f37f524a00ull, 0x341758904b6b0800ull, 0x3477b78023dd8e00ull, 0x28d3a20323692800ull,
    0x1cbad7a3915b1200ull, 0x2c23b4b6f83e9a00ull, 0x3929dec15a6c6400ull, 0x4599fa9edada1c00ull, 0x5143344e0a505000ull, 0x59cab875aa221c00ull, 0x5942f5de8b02f400ull, 0x44aaf18931ba6000ull};
  return t[k];
}
__host__ __device__ constexpr bool irkgl_w_neg(int k) { return (0x555555555555554aull >> k) & 1ull; }
__host__ __device__ constexpr unsigned irkgl_w_bias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x60000000u, 0x8a7cec8eu, 0x000000aeu,
    0x00000000u, 0xe0000000u, 0x1a460c92u, 0x000019c3u,
    0x00000000u, 0x20000000u, 0x352c3db0u, 0x0001146eu,
    0x00000000u, 0x40000000u, 0x27db7de9u, 0x0007a722u,
    0x00000000u, 0x00000000u, 0x890484a6u, 0x002670fcu,
    0x00000000u, 0x00000000u, 0x851780a8u, 0x00852432u,
    0x00000000u, 0x00000000u, 0x354bd4a0u, 0x013a11beu,
    0x00000000u, 0x00000000u, 0x65bb4f00u, 0x01f90f18u};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned irkgl_w_rbias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x60000000u, 0x458f730bu, 0x000003a6u,
    0x00000000u, 0xe0000000u, 0x061206d9u, 0x00019812u,
    0x00000000u, 0x20000000u, 0xd907ad1eu, 0x00246176u,
    0x00000000u, 0x40000000u, 0x5fd19f7bu, 0x01bd0efau,
    0x00000000u, 0x00000000u, 0xc7c8ce06u, 0x0c784bbeu,
    0x00000000u, 0x00000000u, 0x2986bd68u, 0x367fe150u,
    0x00000000u, 0x00000000u, 0x656f91a0u, 0x94c6d34eu,
    0x00000000u, 0x00000000u, 0xe6d60900u, 0x0263efa9u};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned long long irkgl_mu_mag(int k) {
  constexpr unsigned long long t[64] = {
    0x2000000000000000ull, 0x053dc45f0fb7e400ull, 0x02900f45cadc3200ull, 0x019508d6ef38f800ull, 0x0116233b3721e800ull, 0x00c84f3351f0c400ull, 0x008f56260a46dc00ull, 0x0059d49088d1bc00ull,
    0x453dc45f0fb7e400ull, 0x2000000000000000ull, 0x0590bc29fdea2400ull, 0x02e050beedc58e00ull, 0x01d7333dc6adb000ull, 0x0147f5eb23ba1800ull, 0x00e6982090663000ull, 0x008f56260a46dc00ull,
    0x3d6ff0ba3523ce00ull, 0x4590bc29fdea2400ull, 0x2000000000000000ull, 0x05a3545715663000ull, 0x02f45ffe65639c00ull, 0x01e507a4a9897800ull, 0x0147f5eb23ba1800ull, 0x00c84f3351f0c400ull,
    0x419508d6ef38f800ull, 0x3d1faf41123a7200ull, 0x45a3545715663000ull, 0x2000000000000000ull, 0x05a77ad9ea505800ull, 0x02f45ffe65639c00ull, 0x01d7333dc6adb000ull, 0x0116233b3721e800ull,
    0x3ee9dcc4c8de1800ull, 0x41d7333dc6adb000ull, 0x3d0ba0019a9c6400ull, 0x45a77ad9ea505800ull, 0x2000000000000000ull, 0x05a3545715663000ull, 0x02e050beedc58e00ull, 0x019508d6ef38f800ull,
    0x40c84f3351f0c400ull, 0x3eb80a14dc45e800ull, 0x41e507a4a9897800ull, 0x3d0ba0019a9c6400ull, 0x45a3545715663000ull, 0x2000000000000000ull, 0x0590bc29fdea2400ull, 0x02900f45cadc3200ull,
    0x3f70a9d9f5b92400ull, 0x40e6982090663000ull, 0x3eb80a14dc45e800ull, 0x41d7333dc6adb000ull, 0x3d1faf41123a7200ull, 0x4590bc29fdea2400ull, 0x2000000000000000ull, 0x053dc45f0fb7e400ull,
    0x4059d49088d1bc00ull, 0x3f70a9d9f5b92400ull, 0x40c84f3351f0c400ull, 0x3ee9dcc4c8de1800ull, 0x419508d6ef38f800ull, 0x3d6ff0ba3523ce00ull, 0x453dc45f0fb7e400ull, 0x2000000000000000ull};
  return t[k];
}
__host__ __device__ constexpr bool irkgl_mu_neg(int k) { return (0x008040a050a854aaull >> k) & 1ull; }
__host__ __device__ constexpr unsigned irkgl_mu_bias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x00000000u, 0xa6523340u, 0x038812f5u,
    0x00000000u, 0x00000000u, 0xdad00c40u, 0x0c34db34u,
    0x00000000u, 0x00000000u, 0xd5696740u, 0x13dd8af3u,
    0x00000000u, 0x00000000u, 0x204c22c0u, 0x1c1c7c32u,
    0x00000000u, 0x00000000u, 0xdfb3dd40u, 0x23e383cdu,
    0x00000000u, 0x00000000u, 0x2a9698c0u, 0x2c22750cu,
    0x00000000u, 0x00000000u, 0x252ff3c0u, 0x33cb24cbu,
    0x00000000u, 0x00000000u, 0x59adccc0u, 0x3c77ed0au};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned irkgl_mu_rbias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x00000000u, 0x80058f40u, 0x0b7d03efu,
    0x00000000u, 0x00000000u, 0x2fce1040u, 0x148362bdu,
    0x00000000u, 0x00000000u, 0xe649d340u, 0x1c2e3622u,
    0x00000000u, 0x00000000u, 0xd14a2ac0u, 0x239b2a49u,
    0x00000000u, 0x00000000u, 0xe4530540u, 0x2b1be0fbu,
    0x00000000u, 0x00000000u, 0x2880bcc0u, 0x31b33136u,
    0x00000000u, 0x00000000u, 0x34e7d7c0u, 0x3908e92au,
    0x00000000u, 0x00000000u, 0x59adccc0u, 0x3c77ed0au};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned long long irkgl_nu_mag(int k) {
  constexpr unsigned long long t[64] = {
    0x00000304af05335dull, 0x000004cee5e85265ull, 0x000006b2263255e8ull, 0x0000093c4f7f2a07ull, 0x00000d455a464894ull, 0x000014d7d24c5f3dull, 0x000026b318d27721ull, 0x0000624cb581af54ull,
    0x00005e5d327d13c6ull, 0x0000958c7a3a698bull, 0x0000ce034147aca2ull, 0x000116738b3c41eaull, 0x000180f36d71f5b7ull, 0x00022d7cf4470f8cull, 0x00034eea561590deull, 0x000497cfa1c1ab8aull,
    0x0006261b0b04b0c4ull, 0x0009aabc6f1e6910ull, 0x000d194ed2487393ull, 0x00113010d1cfa812ull, 0x00168ab75a434d50ull, 0x001d9f91454f1d2full, 0x002562e0e55a9c8cull, 0x00255c4248899f08ull,
    0x003dcd76edd8c22eull, 0x00605b25dd363910ull, 0x008064c1976a4aa8ull, 0x00a3b0a85bc2c740ull, 0x00ccb9e177b68498ull, 0x00f919c097f0a628ull, 0x011742225b338350ull, 0x00f098102edd3a78ull,
    0x017e882400ddbeb0ull, 0x025028aae6b48a60ull, 0x030a0ce50a12a7a0ull, 0x03c939cf73e18e00ull, 0x04918fe99a18cb00ull, 0x05463f9e64f478c0ull, 0x0584176604f6a0c0ull, 0x046e273f473d6800ull,
    0x05d53bec1d068100ull, 0x08fb13c1948c2180ull, 0x0bad7ca862149880ull, 0x0e4e6f2510cecb00ull, 0x10d830ff6f109500ull, 0x12ce00c0e553f900ull, 0x12e3a51501d4a200ull, 0x0ea2f4a108ac7a00ull,
    0x0eb620c574b12b80ull, 0x16919f4883411400ull, 0x1d2501238d6f6200ull, 0x235254279047bc00ull, 0x28f3e55e6a901200ull, 0x2ccf159d0d3c7600ull, 0x2bffdd0003b34800ull, 0x2174f577827a1a00ull,
    0x1870ed3f67fa8000ull, 0x256c0852114f3e00ull, 0x3025b29549f0d600ull, 0x3a0510ad15724c00ull, 0x42bc2a18b948d400ull, 0x4848448ba3f0f400ull, 0x4631a911ccff9c00ull, 0x34e7671642f4cc00ull};
  return t[k];
}
__host__ __device__ constexpr bool irkgl_nu_neg(int k) { return (0x5555555555555555ull >> k) & 1ull; }
__host__ __device__ constexpr unsigned irkgl_nu_bias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x60000000u, 0x0e9ca840u, 0x000008f0u,
    0x00000000u, 0xc0000000u, 0xcc8663f1u, 0x00004ea1u,
    0x00000000u, 0xc0000000u, 0xd63b77e4u, 0x0001d533u,
    0x00000000u, 0x40000000u, 0x54f33986u, 0x000971ecu,
    0x00000000u, 0x00000000u, 0xeb9904e2u, 0x0025f19fu,
    0x00000000u, 0x00000000u, 0xf46b61e0u, 0x006f7d33u,
    0x00000000u, 0x00000000u, 0xa65b6f10u, 0x00eb2347u,
    0x00000000u, 0x00000000u, 0x3aae7080u, 0x01638a34u};
  return t[i * 4 + w];
}
__host__ __device__ constexpr unsigned irkgl_nu_rbias(int i, int w) {
  constexpr unsigned t[32] = {
    0x00000000u, 0x60000000u, 0x56ecf13au, 0x0000469fu,
    0x00000000u, 0xc0000000u, 0x03d2aaeeu, 0x00064ae0u,
    0x00000000u, 0xc0000000u, 0xf3268617u, 0x00510235u,
    0x00000000u, 0x40000000u, 0xad204e44u, 0x02aba028u,
    0x00000000u, 0x00000000u, 0x9598d6f2u, 0x0ec42df8u,
    0x00000000u, 0x00000000u, 0xe46bb260u, 0x35ae0bdcu,
    0x00000000u, 0x00000000u, 0x16bf5690u, 0x81ba078fu,
    0x00000000u, 0x00000000u, 0x72e23680u, 0xd2e7fd33u};
  return t[i * 4 + w];
}

// Fixed-point sine and cosine (see gen_tables.sincos_tables): 2/pi * 2^128 as
// two 64-bit words; Taylor coefficients of sin(pi/2 f)/f and cos(pi/2 f) in z = f^2,
// scaled by 2^62, constant term first.
#define IRKGL_SINCOS_TERMS 11
#define IRKGL_TWO_OVER_PI_HI 0xa2f9836e4e441529ULL
#define IRKGL_TWO_OVER_PI_LO 0xfc2757d1f534ddc1ULL
__host__ __device__ constexpr long long irkgl_sin_coef(int k) {
  constexpr long long t[11] = {
    7244019458077122842LL,
    -2978983596875621757LL,
    367517370231208053LL,
    -21590780087563799LL,
    739904368663792LL,
    -16596735030340LL,
    262505142787LL,
    -3084311801LL,
    27978803LL,
    -201857LL,
    1186LL};
  return t[k];
}
__host__ __device__ constexpr long long irkgl_cos_coef(int k) {
  constexpr long long t[11] = {
    4611686018427387904LL,
    -5689439577989151081LL,
    1169844122888618931LL,
    -96215822532083616LL,
    4239339756772701LL,
    -116223906447658LL,
    2172507535204LL,
    -29453008147LL,
    302801603LL,
    -2441611LL,
    15854LL};
  return t[k];
}
